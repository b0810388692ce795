// C interface (include/psst.h): validation, device layout, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/psst.h"
#include "psst_internal.h"
#include "psst_syn.cuh"

using psst::NetView;

namespace {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    if (e == cudaErrorMemoryAllocation)
        return fail(PSST_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    return fail(PSST_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Steady state of a gate at V (FP64 host arithmetic; used for the default
// initial state only).
void rest_gates(double V, double out[3]) {
    auto ratio = [](double u) { return u == 0.0 ? 1.0 : u / -std::expm1(-u); };
    const double am = ratio((V + 40.0) / 10.0), bm = 4.0 * std::exp(-(V + 65.0) / 18.0);
    const double ah = 0.07 * std::exp(-(V + 65.0) / 20.0), bh = 1.0 / (1.0 + std::exp(-(V + 35.0) / 10.0));
    const double an = 0.1 * ratio((V + 55.0) / 10.0), bn = 0.125 * std::exp(-(V + 65.0) / 80.0);
    out[0] = am / (am + bm);
    out[1] = ah / (ah + bh);
    out[2] = an / (an + bn);
}

}  // namespace

struct SmemCaps {
    int max_dyn;   // largest dynamic shared memory of one CTA
    int per_sm;    // shared memory of one SM
    int per_cta;   // per-CTA overhead: static shared memory + reserved
};

// What the CTA-mode planner needs, kept so that it can run again when the
// gate uniformity of a network changes (psst_set_state).
struct PlanInput {
    int n_nets = 0, nt = 0, user_K = 0, user_block = 0;
    int min_cl = 1;              // smallest cluster for networks of at least 2 * min_cl neurons
    bool tune_cl = true;         // psst_autotune may choose min_cl
    bool force_synapse_gates = false;
    std::vector<int> net_off, n1, n2;
    std::vector<int> tcnt;       // [N][nt] synapses of each type per row
    std::vector<int> pair_off;   // [n_nets + 1] used (presynaptic neuron, type) pairs of the networks
    std::vector<long long> net_syn;
    std::vector<uint8_t> flags;  // NET_HAS2 | NET_PAIR per network
};

struct psst_net {
    int device = 0;
    PlanInput pin;
    NetView v{};
    psst::GridView gv{};
    std::vector<psst::ClassLaunch> classes;  // CTA mode: one launch per size class
    std::vector<void *> allocs;
    long long step = 0;       // global step index of the current state
    long long rec_reset = 0;  // step at which the record ring was last reset
    int mode = PSST_MODE_CTA;
    int block = 0, K = 0, smem = 0, grid = 0;
    int n_smem = 0, n_global = 0;
    int launches = 0;
    int n_ntypes = 0;
    int max_dyn = 0;
    SmemCaps caps{};
    // adjoint plan and scratch (allocated on the first psst_adjoint)
    std::vector<int> adj_K, adj_items;
    int adj_smem = 0;
    int *d_adjK = nullptr, *d_adjI = nullptr, *d_adjKC = nullptr, *d_adjCI = nullptr;
    int *d_cib = nullptr, *d_ck = nullptr;  // column plan: items of each pair, synapse of each slot
    unsigned short *d_crow = nullptr;       // row of each column slot
    long long *d_segoff = nullptr, *d_cslotoff = nullptr, *d_ciboff = nullptr;
    float *adj_seg = nullptr, *adj_gy0 = nullptr;
    float4 *adj_gpart = nullptr;
    double *adj_gtot = nullptr;
    double *adj_gpn = nullptr;
    long long adj_seg_cap = 0;
    int adj_ckpt_every = 0;
    // checkpoints recorded by psst_integrate for a later psst_adjoint
    int rec_ck_every = 0;
    int rec_ck_spacing = 0;  // checkpoint spacing of the valid recording
    long long rec_ck_cap = 0;  // floats of each checkpoint buffer
    long long rec_ck_cap_steps = 0, rec_ck_start = 0, rec_ck_nsteps = 0;
    bool rec_ck_valid = false;
    float *rec_ck = nullptr;
    float *rec_ck_lo = nullptr;  // the recorded states' remainders
    // CUDA-graph replay of one integrate chunk
    bool graph_mode = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    long long graph_nsteps = 0;
    long long graph_step0 = 0;  // first step of the captured call
    int graph_launches = 0;
    float *tune_buf = nullptr;  // state copy for autotuning trials
    uint8_t *d_check = nullptr; // per-network result of the pair-uniformity check
    // CTA mode: networks without synapses, integrated one thread per neuron
    int *d_ind_neuron = nullptr, *d_ind_net = nullptr;
    int n_ind_neurons = 0, n_ind_nets = 0;

    void drop_graph() {
        if (graph_exec) cudaGraphExecDestroy(graph_exec);
        if (graph) cudaGraphDestroy(graph);
        graph_exec = nullptr;
        graph = nullptr;
        graph_nsteps = 0;
    }

    psst_allocator user_alloc{};  // the caller's device-memory provider, or all NULL (cudaMalloc)

    template <class T>
    cudaError_t alloc(T **p, size_t count) {
        void *q = nullptr;
        const size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
        cudaError_t e = cudaSuccess;
        if (user_alloc.alloc) {
            q = user_alloc.alloc(bytes, user_alloc.ctx);
            if (!q) {
                e = cudaErrorMemoryAllocation;
            } else if ((uintptr_t)q & 255u) {  // the kernels' vector and 64-bit accesses need the documented alignment
                user_alloc.free(q, user_alloc.ctx);
                q = nullptr;
                e = cudaErrorMisalignedAddress;
            }
        } else {
            e = cudaMalloc(&q, bytes);
        }
        if (e == cudaSuccess) allocs.push_back(q);
        *p = (T *)q;
        return e;
    }
    // CTA mode: one stream per size class; an integrate call forks them off
    // the caller's stream and joins them back, so the classes' launches run
    // concurrently and one class's tail overlaps the others' work
    std::vector<cudaStream_t> class_streams;
    std::vector<cudaEvent_t> class_events;  // [0] fork, [1 + c] join of class c

    void drop_streams() {
        for (cudaStream_t s : class_streams) cudaStreamDestroy(s);
        for (cudaEvent_t e : class_events) cudaEventDestroy(e);
        class_streams.clear();
        class_events.clear();
    }
    cudaError_t make_streams(size_t n) {
        if (class_streams.size() == n) return cudaSuccess;
        drop_streams();
        for (size_t i = 0; i < n; ++i) {
            cudaStream_t s;
            cudaError_t e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
            if (e != cudaSuccess) return e;
            class_streams.push_back(s);
        }
        for (size_t i = 0; i <= n; ++i) {
            cudaEvent_t ev;
            cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) return e;
            class_events.push_back(ev);
        }
        return cudaSuccess;
    }
    void release() {
        drop_graph();
        drop_streams();
        for (void *p : allocs) {
            if (user_alloc.free) user_alloc.free(p, user_alloc.ctx);
            else cudaFree(p);
        }
        allocs.clear();
    }
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (dev >= 0 && dev != prev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

template <class T>
cudaError_t upload(psst_net *h, T **dst, const T *src, size_t count) {
    cudaError_t e = h->alloc(dst, count);
    if (e != cudaSuccess || count == 0) return e;
    return cudaMemcpy(*dst, src, count * sizeof(T), cudaMemcpyHostToDevice);
}

int validate(const psst_network_desc *d) {
    if (!d) return fail(PSST_ERR_INVALID_ARG, "desc is NULL");
    if (d->n_nets < 1) return fail(PSST_ERR_INVALID_ARG, "n_nets must be >= 1 (got %d)", d->n_nets);
    if (!d->net_neuron_off || !d->neuron_type || !d->neuron_params || !d->row_ptr || !d->i_const ||
        !d->syn_params)
        return fail(PSST_ERR_INVALID_ARG, "a required array pointer is NULL");
    if (d->net_neuron_off[0] != 0) return fail(PSST_ERR_INVALID_ARG, "net_neuron_off[0] must be 0");
    for (int b = 0; b < d->n_nets; ++b)
        if (d->net_neuron_off[b + 1] < d->net_neuron_off[b])
            return fail(PSST_ERR_INVALID_ARG, "net_neuron_off decreases at net %d", b);
    const long long N = d->net_neuron_off[d->n_nets];
    if (N < 1) return fail(PSST_ERR_INVALID_ARG, "the batch has no neurons");
    if (d->n_neuron_types < 1) return fail(PSST_ERR_INVALID_ARG, "n_neuron_types must be >= 1");
    if (d->n_syn_types < 1 || d->n_syn_types > PSST_MAX_SYN_TYPES)
        return fail(PSST_ERR_INVALID_ARG, "n_syn_types must be in 1..%d", PSST_MAX_SYN_TYPES);
    if (!(d->dt > 0.0f) || !std::isfinite(d->dt)) return fail(PSST_ERR_INVALID_ARG, "dt must be > 0");
    if (d->noise_thresh > (1u << 24)) return fail(PSST_ERR_INVALID_ARG, "noise_thresh must be <= 2^24");
    if (!std::isfinite(d->noise_amp)) return fail(PSST_ERR_INVALID_ARG, "noise_amp not finite");
    if (d->rec_stride < 0) return fail(PSST_ERR_INVALID_ARG, "rec_stride must be >= 0");
    if (d->rec_stride > 0 && d->rec_capacity < 1)
        return fail(PSST_ERR_INVALID_ARG, "rec_capacity must be >= 1 when recording");
    if (d->pulse_amp && (!d->pulse_on || !d->pulse_off))
        return fail(PSST_ERR_INVALID_ARG, "pulse_amp given without pulse_on/pulse_off");
    if (d->block_threads && (d->block_threads % 32 || d->block_threads < 32 || d->block_threads > 1024))
        return fail(PSST_ERR_INVALID_ARG, "block_threads must be a multiple of 32 in 32..1024");
    if (d->item_chunks < 0 || d->item_chunks > 64)
        return fail(PSST_ERR_INVALID_ARG, "item_chunks must be in 0..64");
    for (int t = 0; t < d->n_neuron_types; ++t) {
        const float *p = d->neuron_params + (size_t)t * PSST_NEURON_NPARAM;
        for (int x = 0; x < PSST_NEURON_NPARAM; ++x)
            if (!std::isfinite(p[x])) return fail(PSST_ERR_INVALID_ARG, "neuron type %d param %d not finite", t, x);
        if (!(p[0] > 0.0f)) return fail(PSST_ERR_INVALID_ARG, "neuron type %d: C must be > 0", t);
    }
    for (int t = 0; t < d->n_syn_types; ++t) {
        const float *q = d->syn_params + (size_t)t * PSST_SYN_NPARAM;
        for (int x = 0; x < PSST_SYN_NPARAM; ++x)
            if (!std::isfinite(q[x])) return fail(PSST_ERR_INVALID_ARG, "synapse type %d param %d not finite", t, x);
        if (q[0] != 0.0f && q[0] != 1.0f) return fail(PSST_ERR_INVALID_ARG, "synapse type %d: kind must be 0 or 1", t);
        if (!(q[8] > 0.0f)) return fail(PSST_ERR_INVALID_ARG, "synapse type %d: Kp must be > 0", t);
        if (q[0] == 1.0f && !(q[5] > 0.0f)) return fail(PSST_ERR_INVALID_ARG, "synapse type %d: Kd must be > 0", t);
    }
    if (d->row_ptr[0] != 0) return fail(PSST_ERR_INVALID_ARG, "row_ptr[0] must be 0");
    for (long long i = 0; i < N; ++i)
        if (d->row_ptr[i + 1] < d->row_ptr[i]) return fail(PSST_ERR_INVALID_ARG, "row_ptr decreases at row %lld", i);
    const long long S = d->row_ptr[N];
    if (S > 0 && (!d->pre || !d->weight || !d->syn_type))
        return fail(PSST_ERR_INVALID_ARG, "synapse arrays are NULL but row_ptr[N] = %lld", S);
    for (long long i = 0; i < N; ++i) {
        if (d->neuron_type[i] < 0 || d->neuron_type[i] >= d->n_neuron_types)
            return fail(PSST_ERR_INVALID_ARG, "neuron_type[%lld] out of range", i);
        if (!std::isfinite(d->i_const[i])) return fail(PSST_ERR_INVALID_ARG, "i_const[%lld] not finite", i);
        if (d->pulse_amp && !std::isfinite(d->pulse_amp[i]))
            return fail(PSST_ERR_INVALID_ARG, "pulse_amp[%lld] not finite", i);
    }
    for (int b = 0; b < d->n_nets; ++b) {
        const long long n0 = d->net_neuron_off[b], n1 = d->net_neuron_off[b + 1];
        const long long nb = n1 - n0;
        if (nb * d->n_syn_types >= (1LL << 24))
            return fail(PSST_ERR_UNSUPPORTED, "net %d: %lld neurons x %d synapse types exceeds 2^24", b, nb,
                        d->n_syn_types);
        for (long long k = d->row_ptr[n0]; k < d->row_ptr[n1]; ++k) {
            if (d->pre[k] < 0 || d->pre[k] >= nb)
                return fail(PSST_ERR_INVALID_ARG, "pre[%lld] = %d outside its network (size %lld)", k, d->pre[k], nb);
            if (d->syn_type[k] < 0 || d->syn_type[k] >= d->n_syn_types)
                return fail(PSST_ERR_INVALID_ARG, "syn_type[%lld] out of range", k);
            if (!std::isfinite(d->weight[k])) return fail(PSST_ERR_INVALID_ARG, "weight[%lld] not finite", k);
        }
    }
    if (d->init_state) {
        const long long dim = 4 * N + 2 * S;
        for (long long i = 0; i < dim; ++i)
            if (!std::isfinite(d->init_state[i])) return fail(PSST_ERR_INVALID_ARG, "init_state[%lld] not finite", i);
    }
    if (d->mode < PSST_MODE_AUTO || d->mode > PSST_MODE_GRID) return fail(PSST_ERR_INVALID_ARG, "unknown mode");
    if (d->gate_mode < 0 || d->gate_mode > 1) return fail(PSST_ERR_INVALID_ARG, "gate_mode must be 0 or 1");
    if (d->min_cluster != 0 && d->min_cluster != 1 && d->min_cluster != 2 && d->min_cluster != 4)
        return fail(PSST_ERR_INVALID_ARG, "min_cluster must be 0, 1, 2 or 4");
    if (d->method != PSST_METHOD_RK4 && d->method != PSST_METHOD_EULER && d->method != PSST_METHOD_TABLEAU)
        return fail(PSST_ERR_INVALID_ARG,
                    "method must be PSST_METHOD_RK4 (0), PSST_METHOD_EULER (1) or PSST_METHOD_TABLEAU (2)");
    if (d->method == PSST_METHOD_TABLEAU) {
        if (d->rk_stages < 1 || d->rk_stages > 4) return fail(PSST_ERR_INVALID_ARG, "rk_stages must be 1..4");
        bool any = false;
        for (int q = 0; q < d->rk_stages; ++q) {
            if (!std::isfinite(d->rk_b[q]) || (q > 0 && !std::isfinite(d->rk_a[q - 1])))
                return fail(PSST_ERR_INVALID_ARG, "rk_a / rk_b must be finite (stage %d)", q + 1);
            any |= d->rk_b[q] != 0.0f;
        }
        if (!any) return fail(PSST_ERR_INVALID_ARG, "rk_b must not be all zero");
    }
    return PSST_OK;
}

// Per-row counts of first- and second-order synapses and of each synapse
// type, and which networks hold second-order synapses.
void row_counts(const psst_network_desc *d, std::vector<int> &n1, std::vector<int> &n2, std::vector<int> &tcnt,
                std::vector<uint8_t> &has2) {
    const long long N = d->net_neuron_off[d->n_nets];
    const int nt = d->n_syn_types;
    n1.assign((size_t)N, 0);
    n2.assign((size_t)N, 0);
    tcnt.assign((size_t)N * nt, 0);
    has2.assign((size_t)d->n_nets, 0);
    for (int b = 0; b < d->n_nets; ++b) {
        for (long long i = d->net_neuron_off[b]; i < d->net_neuron_off[b + 1]; ++i) {
            for (long long k = d->row_ptr[i]; k < d->row_ptr[i + 1]; ++k) {
                if (d->syn_params[(size_t)d->syn_type[k] * PSST_SYN_NPARAM] != 0.0f) ++n2[i];
                else ++n1[i];
                ++tcnt[(size_t)i * nt + d->syn_type[k]];
            }
            if (n2[i]) has2[b] = 1;
        }
    }
}

// Split rows [0, n) with per-row cost into `parts` contiguous blocks of
// about equal cost.  split has parts + 1 entries.
void balanced_split(const std::vector<double> &cost, int parts, std::vector<int> &split) {
    const int n = (int)cost.size();
    std::vector<double> pref((size_t)n + 1, 0.0);
    for (int i = 0; i < n; ++i) pref[i + 1] = pref[i] + cost[i];
    split.assign((size_t)parts + 1, 0);
    split[parts] = n;
    for (int c = 1; c < parts; ++c) {
        const double target = pref[n] * c / parts;
        int lo = split[c - 1], hi = n;
        while (lo < hi) {
            const int mid = (lo + hi) / 2;
            if (pref[mid] < target) lo = mid + 1;
            else hi = mid;
        }
        split[c] = lo;
    }
}


int smem_caps(int dev, SmemCaps *c) {
    int optin = 0, per_sm = 0, reserved = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess)
        return fail(PSST_ERR_CUDA, "cannot query shared memory sizes of device %d", dev);
    const int stat = psst::cta_static_smem() + 64;  // static table + small shared variables
    c->max_dyn = optin - stat;
    c->per_sm = per_sm;
    c->per_cta = stat + reserved;
    return PSST_OK;
}

// 4-synapse chunks per work item: about 768 threads' worth of items for the
// largest CTA share, 1..8 (or the caller's choice).
int choose_K(long long chunks, int user) {
    if (user > 0) return user;
    const long long k = (chunks + 767) / 768;
    return (int)std::max(1LL, std::min(8LL, k));
}

struct Share {  // one CTA's share of a network
    int r0, r1, items1, items2;
    long long chunks;
};

// Shares of `parts` CTAs over rows [0, n) (row i of the network at n1[i],
// n2[i]) and the work-item size.  With tcnt (per row, synapses of each of
// the nt types) the items are the per-pair variant's typed items, all in
// list 1.
void make_shares(const int *n1, const int *n2, const int *tcnt, int nt, int n, int parts, int user_K,
                 std::vector<Share> &sh, int *K) {
    auto row_chunks = [&](int i) -> long long {
        if (!tcnt) return (n1[i] + 3) / 4 + (n2[i] + 3) / 4;
        long long c = 0;
        for (int t = 0; t < nt; ++t) c += (tcnt[(size_t)i * nt + t] + 3) / 4;
        return c;
    };
    std::vector<double> cost((size_t)n);
    for (int i = 0; i < n; ++i) cost[i] = (double)row_chunks(i) + 2.0;
    std::vector<int> split;
    balanced_split(cost, parts, split);
    sh.assign((size_t)parts, Share{});
    long long worst = 0;
    for (int q = 0; q < parts; ++q) {
        sh[q].r0 = split[q];
        sh[q].r1 = split[q + 1];
        for (int i = split[q]; i < split[q + 1]; ++i) sh[q].chunks += row_chunks(i);
        worst = std::max(worst, sh[q].chunks);
    }
    *K = choose_K(worst, user_K);
    for (int q = 0; q < parts; ++q) {
        sh[q].items1 = sh[q].items2 = 0;
        for (int i = split[q]; i < split[q + 1]; ++i) {
            if (tcnt) {
                sh[q].items1 += psst::typed_row_items(tcnt + (size_t)i * nt, nt, *K);
            } else {
                sh[q].items1 += psst::part_items(n1[i], *K);
                sh[q].items2 += psst::part_items(n2[i], *K);
            }
        }
    }
}

// Dynamic shared memory of one CTA of a network of N neurons in CTA mode.
long long cta_share_bytes(int N, int nt, int used_pairs, bool has2, bool pair, const Share &s, int K,
                          int rep = 1) {
    const psst::NeuronLayout L = psst::make_nlayout(s.r1 - s.r0, N, pair ? used_pairs : N * nt, has2, pair, rep);
    return L.syn + (pair ? psst::items_smem_bytes_pair(s.items1, K, s.r1 - s.r0)
                         : psst::items_smem_bytes(s.items1, s.items2, K, s.r1 - s.r0, has2));
}

// CTAs of `need` bytes of dynamic shared memory that one SM holds (1..4).
int ctas_per_sm(const SmemCaps &caps, long long need) {
    return (int)std::max(1LL, std::min(4LL, (long long)caps.per_sm / (need + caps.per_cta)));
}

// Smallest cluster size (1, 2, 4) whose CTAs all fit; 0 if none.  Per-pair
// gates: the gate table gets the most copies (up to 32) that leave the CTAs
// per SM as they are with one copy.
int plan_network(const PlanInput &in, int b, const SmemCaps &caps, psst::NetPlan *pl, long long *need) {
    const int n0 = in.net_off[b], N = in.net_off[b + 1] - n0, nt = in.nt;
    const bool has2 = in.flags[b] & psst::NET_HAS2, pair = in.flags[b] & psst::NET_PAIR;
    const std::vector<int> &n1 = in.n1, &n2 = in.n2;
    const int *tc = pair ? in.tcnt.data() + (size_t)n0 * nt : nullptr;
    // a network spread over a larger cluster than it needs keeps the work-item
    // size of one CTA, so the summation order (and every result) is the same
    int user_K = in.user_K;
    if (in.min_cl > 1 && N >= 2 * in.min_cl && user_K == 0) {
        std::vector<Share> sh1;
        make_shares(n1.data() + n0, n2.data() + n0, tc, nt, N, 1, 0, sh1, &user_K);
    }
    for (int cl = 1; cl <= PSST_MAX_CL; cl *= 2) {
        if (cl > 1 && N < 2 * cl) break;
        if (cl < in.min_cl && N >= 2 * in.min_cl) continue;  // spread over a larger cluster
        std::vector<Share> sh;
        int K = 1;
        make_shares(n1.data() + n0, n2.data() + n0, tc, nt, N, cl, user_K, sh, &K);
        long long worst = 0;
        const int used = in.pair_off[b + 1] - in.pair_off[b];
        for (int q = 0; q < cl; ++q) worst = std::max(worst, cta_share_bytes(N, nt, used, has2, pair, sh[q], K));
        if (worst <= caps.max_dyn) {
            std::memset(pl, 0, sizeof *pl);
            if (pair) {
                const int base = ctas_per_sm(caps, worst);
                for (int lrep = 5; lrep > 0; --lrep) {
                    long long w = 0;
                    for (int q = 0; q < cl; ++q)
                        w = std::max(w, cta_share_bytes(N, nt, used, has2, pair, sh[q], K, 1 << lrep));
                    if (w <= caps.max_dyn && ctas_per_sm(caps, w) >= base) {
                        pl->lrep = lrep;
                        worst = w;
                        break;
                    }
                }
            }
            pl->K = K;
            for (int q = 0; q < cl; ++q) {
                pl->split[q] = sh[q].r0;
                pl->n1[q] = sh[q].items1;
                pl->n2[q] = sh[q].items2;
            }
            pl->split[cl] = N;
            *need = worst;
            return cl;
        }
    }
    return 0;
}

// Per network: do all gates of each (presynaptic neuron, type) pair hold the
// same value in the state y ([V, m, h, n, r, s], host memory; NULL = rest,
// all gates 0)?
std::vector<uint8_t> uniform_pairs(const float *y, const PlanInput &in, const int64_t *row_ptr, const int32_t *pre,
                                   const int32_t *syn_type, long long N, long long S) {
    std::vector<uint8_t> ok((size_t)in.n_nets, 1);
    if (!y) return ok;
    const float *r = y + 4 * N, *s = y + 4 * N + S;
    for (int b = 0; b < in.n_nets; ++b) {
        const int n0 = in.net_off[b], nb = in.net_off[b + 1] - n0;
        std::vector<float> rr((size_t)nb * in.nt), ss((size_t)nb * in.nt);
        std::vector<uint8_t> seen((size_t)nb * in.nt, 0);
        for (long long k = row_ptr[n0]; k < row_ptr[n0 + nb] && ok[b]; ++k) {
            const size_t p = (size_t)pre[k] * in.nt + syn_type[k];
            if (!seen[p]) {
                seen[p] = 1;
                rr[p] = r[k];
                ss[p] = s[k];
            } else if (std::memcmp(&rr[p], &r[k], 4) || std::memcmp(&ss[p], &s[k], 4)) {
                ok[b] = 0;
            }
        }
    }
    return ok;
}

// Grid mode, per-pair gates: the compact table index of every
// (presynaptic neuron, type) pair that has a synapse, in pair order, and one
// synapse of each such pair.  Built once from the connectivity.
int grid_pair_tables(psst_net *h, const psst_network_desc *d, cudaError_t *err) {
    const long long N = h->v.N, S = h->v.S;
    const int nt = h->v.n_stypes;
    const long long M = N * nt;
    std::vector<long long> first((size_t)M, -1);
    for (long long k = 0; k < S; ++k) {
        const size_t p = (size_t)d->pre[k] * nt + d->syn_type[k];
        if (first[p] < 0) first[p] = k;
    }
    std::vector<long long> rep;  // in pair order, as the compact index of the network's used pairs
    for (long long p = 0; p < M; ++p)
        if (first[p] >= 0) rep.push_back(first[p]);
    psst::GridView &g = h->gv;
    const long long used = (long long)rep.size();
    g.mt = (int)((used + 3) & ~3LL);
    long long *r = nullptr;
    cudaError_t e = upload(h, &r, rep.data(), rep.size());
    g.used = (int)used;
    if (e == cudaSuccess) e = h->alloc(&g.r0g, (size_t)used);
    if (e == cudaSuccess) e = h->alloc(&g.s0g, (size_t)used);
    if (e == cudaSuccess) e = h->alloc(&g.r0lg, (size_t)used);
    if (e == cudaSuccess) e = h->alloc(&g.s0lg, (size_t)used);
    g.tix = h->v.pair_tix;
    g.rep = r;
    if (e != cudaSuccess) return *err = e, cuda_fail(e, "grid pair tables");
    return PSST_OK;
}

// Grid mode: one contiguous block of rows per CTA with balanced cost, the
// double-buffered gate tables and the barrier words.  Per-pair gates when
// the network's pairs are uniform (flag NET_PAIR) and the compact gate
// table fits in shared memory next to the items; re-run when that changes.
int setup_grid(psst_net *h, const SmemCaps &caps, cudaError_t *err) {
    const PlanInput &in = h->pin;
    const long long N = h->v.N;
    const int nt = h->v.n_stypes;
    const bool has2 = in.flags[0] & psst::NET_HAS2;
    if (N * nt >= 65536)
        return fail(PSST_ERR_UNSUPPORTED, "grid mode: %lld neurons x %d synapse types must stay below 65536", N, nt);
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return *err = e, cuda_fail(e, "device attributes");
    const int parts = (int)std::max<long long>(1, std::min<long long>(sms, (N + 7) / 8));
    psst::GridView &g = h->gv;
    // per-pair plan (typed items next to the compact gate table), else per synapse
    auto plan = [&](bool pair, std::vector<Share> &sh, int *K) -> long long {
        make_shares(in.n1.data(), in.n2.data(), pair ? in.tcnt.data() : nullptr, nt, (int)N, parts, in.user_K, sh,
                    K);
        long long need = 0;
        for (int c = 0; c < parts; ++c) {
            const int n = sh[c].r1 - sh[c].r0;
            const long long bytes =
                pair ? psst::make_nlayout(n, n, n * nt, has2, true, 0).syn + 4LL * g.mt +
                           psst::items_smem_bytes_pair(sh[c].items1, *K, n)
                     : psst::make_nlayout(n, n, n * nt, has2).syn +
                           psst::items_smem_bytes(sh[c].items1, sh[c].items2, *K, n, has2);
            need = std::max(need, bytes);
        }
        return need;
    };
    std::vector<Share> sh;
    int K = 1;
    bool pair = (in.flags[0] & psst::NET_PAIR) && g.tix != nullptr;
    long long need = pair ? plan(true, sh, &K) : 0;
    if (pair && need > caps.max_dyn) pair = false;
    if (!pair) need = plan(false, sh, &K);
    if (need > caps.max_dyn)
        return fail(PSST_ERR_UNSUPPORTED, "grid mode: a block needs %lld B of shared memory (max %d)", need,
                    caps.max_dyn);
    std::vector<int> split((size_t)parts + 1), items((size_t)2 * parts);
    for (int c = 0; c < parts; ++c) {
        split[c] = sh[c].r0;
        items[c] = sh[c].items1;
        items[parts + c] = sh[c].items2;
    }
    split[parts] = (int)N;
    if (!h->block) h->block = 1024;
    h->K = K;
    h->smem = (int)need;
    int per_sm = 0;
    // the kernel attribute is an upper bound shared by every handle's launches
    e = psst::grid_occupancy(h->block, caps.max_dyn, &per_sm);
    if (e != cudaSuccess) return *err = e, cuda_fail(e, "grid occupancy");
    if (per_sm < 1) return fail(PSST_ERR_UNSUPPORTED, "grid mode: a CTA of %d threads does not fit an SM", h->block);
    h->grid = parts;
    if (!g.row_split) {
        int *rs = nullptr, *itd = nullptr;
        e = h->alloc(&rs, split.size());
        if (e == cudaSuccess) e = h->alloc(&itd, items.size());
        if (e == cudaSuccess) e = h->alloc(&g.c1, (size_t)(2 * N * nt));
        if (e == cudaSuccess && has2) e = h->alloc(&g.c2, (size_t)(2 * N * nt));
        if (e == cudaSuccess) e = h->alloc(&g.flag, (size_t)parts * psst::GRID_FLAG_STRIDE);
        if (e == cudaSuccess && g.tix) {
            g.gts = g.used + parts;
            e = h->alloc(&g.gt, (size_t)2 * g.gts);
        }
        g.row_split = rs;
        g.items = itd;
        if (e != cudaSuccess) return *err = e, cuda_fail(e, "grid buffers");
    }
    e = cudaMemcpy((void *)g.row_split, split.data(), split.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy((void *)g.items, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return *err = e, cuda_fail(e, "grid plan upload");
    g.K = K;
    g.pair = pair ? 1 : 0;
    return PSST_OK;
}

// CTA mode: each network's cluster size and work items, size classes by
// cluster size x CTAs per SM, launch lists (largest networks first).
int setup_cta(psst_net *h, const SmemCaps &caps, cudaError_t *err) {
    const PlanInput &in = h->pin;
    const int n_nets = in.n_nets, nt = in.nt;
    const std::vector<int> &n1 = in.n1, &n2 = in.n2;
    h->classes.clear();
    h->n_smem = h->n_global = 0;
    std::vector<psst::NetPlan> plans((size_t)n_nets);
    std::vector<int> cl_of((size_t)n_nets), per_sm((size_t)n_nets);
    std::vector<long long> need((size_t)n_nets);
    std::vector<double> cost((size_t)n_nets);
    std::vector<int> ind_neuron, ind_net;  // neurons of the networks without synapses
    for (int b = 0; b < n_nets; ++b) {
        const int n0 = in.net_off[b], N = in.net_off[b + 1] - n0;
        if (in.net_syn[b] == 0) {  // independent neurons: no size class, no barrier
            cl_of[b] = 0;
            for (int i = n0; i < n0 + N; ++i) {
                ind_neuron.push_back(i);
                ind_net.push_back(b);
            }
            continue;
        }
        if ((long long)N * nt >= 65536)
            return fail(PSST_ERR_UNSUPPORTED, "net %d: %d neurons x %d synapse types must stay below 65536", b, N, nt);
        const int cl = plan_network(in, b, caps, &plans[b], &need[b]);
        if (!cl)
            return fail(PSST_ERR_UNSUPPORTED, "net %d (%d neurons, %lld synapses) does not fit %d CTAs", b, N,
                        in.net_syn[b], PSST_MAX_CL);
        cl_of[b] = cl;
        per_sm[b] = ctas_per_sm(caps, need[b]);
        double c = 0;
        for (int i = n0; i < n0 + N; ++i) c += n1[i] + n2[i] + 30.0;
        cost[b] = c;
    }
    std::vector<int> all_lists;
    std::vector<std::pair<int, int>> ranges;
    for (int cl = PSST_MAX_CL; cl >= 1; cl /= 2) {
        for (int k = 1; k <= 4; ++k) {
            std::vector<int> list;
            for (int b = 0; b < n_nets; ++b)
                if (cl_of[b] == cl && per_sm[b] == k) list.push_back(b);
            if (list.empty()) continue;
            std::stable_sort(list.begin(), list.end(), [&](int a, int b2) { return cost[a] > cost[b2]; });
            psst::ClassLaunch c{};
            c.cl = cl;
            c.n_nets = (int)list.size();
            long long mx = 0;
            for (int b : list) {
                mx = std::max(mx, need[b]);
                c.lrep_cap = std::max(c.lrep_cap, plans[b].lrep);
            }
            c.smem = (int)mx;
            c.block = in.user_block ? in.user_block : ((1024 / k) / 32) * 32;
            ranges.push_back({(int)all_lists.size(), (int)list.size()});
            all_lists.insert(all_lists.end(), list.begin(), list.end());
            h->classes.push_back(c);
        }
    }
    int *dl = nullptr;
    psst::NetPlan *dp = nullptr;
    cudaError_t e = upload(h, &dl, all_lists.data(), all_lists.size());
    if (e == cudaSuccess) e = upload(h, &dp, plans.data(), plans.size());
    for (size_t i = 0; e == cudaSuccess && i < h->classes.size(); ++i) {
        h->classes[i].list = dl + ranges[i].first;
        h->classes[i].plans = dp;
        e = psst::cta_prepare(h->classes[i].cl, caps.max_dyn);
    }
    if (e == cudaSuccess && !ind_neuron.empty() && !h->d_ind_neuron) {
        e = upload(h, &h->d_ind_neuron, ind_neuron.data(), ind_neuron.size());
        if (e == cudaSuccess) e = upload(h, &h->d_ind_net, ind_net.data(), ind_net.size());
    }
    h->n_ind_neurons = (int)ind_neuron.size();
    h->n_ind_nets = 0;
    for (int b = 0; b < n_nets; ++b) h->n_ind_nets += in.net_syn[b] == 0;
    // one stream per launch of an integrate chunk when there are several
    const size_t n_launch = h->classes.size() + (h->n_ind_neurons > 0 ? 1 : 0);
    if (e == cudaSuccess) e = h->make_streams(n_launch > 1 ? n_launch : 0);
    if (e != cudaSuccess) return *err = e, cuda_fail(e, "CTA mode setup");
    h->block = h->classes.empty() ? 0 : h->classes.back().block;
    h->K = plans.empty() ? 0 : plans[h->classes.empty() ? 0 : all_lists.back()].K;
    h->smem = 0;
    h->grid = 0;
    for (auto &c : h->classes) {
        h->smem = std::max(h->smem, c.smem);
        h->grid += c.n_nets * c.cl;
        if (c.cl == 1) h->n_smem += c.n_nets;
        else h->n_global += c.n_nets;
    }
    return PSST_OK;
}

}  // namespace

extern "C" {

const char *psst_error_string(int code) {
    switch (code) {
    case PSST_OK: return "ok";
    case PSST_ERR_INVALID_ARG: return "invalid argument";
    case PSST_ERR_OOM: return "out of device memory";
    case PSST_ERR_CUDA: return "CUDA error";
    case PSST_ERR_NONFINITE: return "state became non-finite";
    case PSST_ERR_TIMEOUT: return "device-wide wait timed out";
    case PSST_ERR_STATE: return "invalid call for the handle's state";
    case PSST_ERR_UNSUPPORTED: return "unsupported network shape for this mode";
    default: return "unknown error";
    }
}

const char *psst_last_error(void) { return g_last_error.c_str(); }

int psst_create_network(const psst_network_desc *d, const psst_allocator *a, psst_net **out) {
    if (!out) return fail(PSST_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int rc = validate(d);
    if (rc) return rc;
    if (a && (!a->alloc || !a->free)) return fail(PSST_ERR_INVALID_ARG, "allocator: alloc and free must both be set");
    int dev = d->device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(PSST_ERR_CUDA, "no CUDA device");
    DeviceGuard guard(dev);

    const int n_nets = d->n_nets, nt = d->n_syn_types;
    const long long N = d->net_neuron_off[n_nets], S = d->row_ptr[N];
    SmemCaps caps;
    rc = smem_caps(dev, &caps);
    if (rc) return rc;

    PlanInput pin;
    pin.n_nets = n_nets;
    pin.nt = nt;
    pin.user_K = d->item_chunks;
    pin.user_block = d->block_threads;
    pin.force_synapse_gates = d->gate_mode == 1;
    pin.min_cl = d->min_cluster > 0 ? d->min_cluster : 1;
    pin.tune_cl = d->min_cluster == 0;
    pin.net_off.assign(d->net_neuron_off, d->net_neuron_off + n_nets + 1);
    pin.net_syn.resize(n_nets);
    for (int b = 0; b < n_nets; ++b)
        pin.net_syn[b] = d->row_ptr[d->net_neuron_off[b + 1]] - d->row_ptr[d->net_neuron_off[b]];
    std::vector<uint8_t> has2;
    row_counts(d, pin.n1, pin.n2, pin.tcnt, has2);
    pin.flags.assign(n_nets, 0);
    {
        const std::vector<uint8_t> uni = uniform_pairs(d->init_state, pin, d->row_ptr, d->pre, d->syn_type, N, S);
        for (int b = 0; b < n_nets; ++b)
            pin.flags[b] = (has2[b] ? psst::NET_HAS2 : 0) |
                           (uni[b] && !pin.force_synapse_gates ? psst::NET_PAIR : 0);
    }
    // compact index of each network's used (presynaptic neuron, type) pairs
    std::vector<int> ptix((size_t)N * nt, -1), pof;
    std::vector<int> &pair_off = pin.pair_off;
    pair_off.assign((size_t)n_nets + 1, 0);
    for (int b = 0; b < n_nets; ++b) {
        const long long n0 = d->net_neuron_off[b], nb = d->net_neuron_off[b + 1] - n0;
        int *tb = ptix.data() + n0 * nt;
        for (long long k = d->row_ptr[n0]; k < d->row_ptr[n0 + nb]; ++k) tb[(size_t)d->pre[k] * nt + d->syn_type[k]] = 0;
        pair_off[b] = (int)pof.size();
        for (long long p = 0; p < nb * nt; ++p)
            if (tb[p] == 0) {
                tb[p] = (int)pof.size() - pair_off[b];
                pof.push_back((int)p);
            }
    }
    pair_off[n_nets] = (int)pof.size();
    bool all_fit = true;
    for (int b = 0; b < n_nets && all_fit; ++b) {
        if (pin.net_syn[b] == 0) continue;  // independent neurons need no shared-memory plan
        psst::NetPlan pl;
        long long need = 0;
        all_fit = plan_network(pin, b, caps, &pl, &need) != 0;
    }
    int mode = d->mode;
    if (mode == PSST_MODE_AUTO) mode = all_fit ? PSST_MODE_CTA : PSST_MODE_GRID;
    if (mode == PSST_MODE_GRID && n_nets != 1)
        return fail(PSST_ERR_UNSUPPORTED, "grid mode integrates a single network (got %d)", n_nets);

    psst_net *h = new psst_net();
    if (a) h->user_alloc = *a;
    h->device = dev;
    h->mode = mode;
    h->pin = pin;
    h->n_ntypes = d->n_neuron_types;
    h->max_dyn = caps.max_dyn;
    h->block = d->block_threads;
    NetView &v = h->v;
    v.n_nets = n_nets;
    v.n_stypes = nt;
    v.N = N;
    v.S = S;
    v.noise_seed = d->noise_seed;
    v.noise_thresh = d->noise_thresh;
    v.noise_amp = d->noise_amp;
    v.dt = d->dt;
    v.method = d->method;
    if (d->method == PSST_METHOD_TABLEAU) {
        // weights relative to the first nonzero b (the classic RK4 tableau
        // then gives the RK4 kernels' own weights 1, 2, 2, 1 and scale 1/6)
        v.rk_ns = d->rk_stages;
        int q0 = 0;
        while (d->rk_b[q0] == 0.0f) ++q0;
        v.rk_beta = d->rk_b[q0];
        for (int q = 0; q < 4; ++q) v.rk_w[q] = q < d->rk_stages ? d->rk_b[q] / v.rk_beta : 0.0f;
        for (int q = 0; q < 3; ++q) v.rk_c[q] = q + 1 < d->rk_stages ? d->rk_a[q] : 0.0f;
    }
    v.rec_stride = d->rec_stride;
    v.rec_cap = d->rec_stride > 0 ? d->rec_capacity : 0;

    std::vector<uint32_t> code((size_t)S);
    for (long long k = 0; k < S; ++k)
        code[k] = ((uint32_t)d->syn_type[k] << 24) | (uint32_t)(d->pre[k] * nt + d->syn_type[k]);


    cudaError_t e = cudaSuccess;
    std::vector<long long> rp(d->row_ptr, d->row_ptr + N + 1);
    std::vector<long long> pon((size_t)n_nets, 0), poff((size_t)n_nets, 0);
    if (d->pulse_amp)
        for (int b = 0; b < n_nets; ++b) pon[b] = d->pulse_on[b], poff[b] = d->pulse_off[b];
#define UP(dst, src, cnt)                                                   \
    do {                                                                    \
        if (e == cudaSuccess) e = upload(h, &(dst), (src), (size_t)(cnt)); \
    } while (0)
    {
        int *p_off, *p_nt;
        long long *p_rp, *p_on, *p_offp;
        uint32_t *p_code;
        float *p_w, *p_np, *p_sp, *p_ic, *p_pa = nullptr;
        uint8_t *p_fl;
        UP(p_off, d->net_neuron_off, n_nets + 1);
        UP(p_rp, rp.data(), N + 1);
        UP(p_code, code.data(), S);
        UP(p_w, d->weight, S);
        UP(p_nt, d->neuron_type, N);
        UP(p_np, d->neuron_params, (size_t)d->n_neuron_types * PSST_NEURON_NPARAM);
        UP(p_sp, d->syn_params, (size_t)nt * PSST_SYN_NPARAM);
        UP(p_ic, d->i_const, N);
        if (d->pulse_amp) UP(p_pa, d->pulse_amp, N);
        UP(p_on, pon.data(), n_nets);
        UP(p_offp, poff.data(), n_nets);
        UP(p_fl, pin.flags.data(), n_nets);
        int *p_tix, *p_pof, *p_poff;
        UP(p_tix, ptix.data(), ptix.size());
        UP(p_pof, pof.data(), pof.size());
        UP(p_poff, pin.pair_off.data(), pin.pair_off.size());
        v.pair_tix = p_tix;
        v.pair_of = p_pof;
        v.pair_off = p_poff;
        v.net_off = p_off;
        v.row_ptr = p_rp;
        v.syn_code = p_code;
        v.weight = p_w;
        v.neuron_type = p_nt;
        v.nparams = p_np;
        v.sparams = p_sp;
        v.i_const = p_ic;
        v.pulse_amp = p_pa;
        v.pulse_on = p_on;
        v.pulse_off = p_offp;
        v.net_flags = p_fl;
    }
#undef UP
    const long long dim = 4 * N + 2 * S;
    if (e == cudaSuccess) e = h->alloc(&v.state, (size_t)dim);
    if (e == cudaSuccess) e = h->alloc(&v.state_lo, (size_t)dim);
    if (e == cudaSuccess) e = cudaMemset(v.state_lo, 0, (size_t)dim * sizeof(float));
    if (e == cudaSuccess && v.rec_cap > 0) e = h->alloc(&v.rec, (size_t)(v.rec_cap * N));
    if (e == cudaSuccess) e = h->alloc(&v.err, 1);
    if (e == cudaSuccess) e = cudaMemset(v.err, 0, sizeof(int));
    if (e == cudaSuccess && v.rec) e = cudaMemset(v.rec, 0, (size_t)v.rec_cap * N * sizeof(float));
    if (e == cudaSuccess) {
        if (d->init_state) {
            e = cudaMemcpy(v.state, d->init_state, (size_t)dim * sizeof(float), cudaMemcpyHostToDevice);
        } else {
            std::vector<float> y((size_t)dim, 0.0f);
            double g[3];
            rest_gates(-65.0, g);
            for (long long i = 0; i < N; ++i) {
                y[i] = -65.0f;
                y[N + i] = (float)g[0];
                y[2 * N + i] = (float)g[1];
                y[3 * N + i] = (float)g[2];
            }
            e = cudaMemcpy(v.state, y.data(), (size_t)dim * sizeof(float), cudaMemcpyHostToDevice);
        }
    }
    if (e != cudaSuccess) {
        h->release();
        delete h;
        return cuda_fail(e, "psst_create_network");
    }
    h->caps = caps;
    if (mode == PSST_MODE_GRID) {
        h->gv.timeout_ns = 2000000000ULL;
        rc = grid_pair_tables(h, d, &e);
        if (!rc) rc = setup_grid(h, caps, &e);
    } else {
        rc = setup_cta(h, caps, &e);
    }
    if (rc) {
        h->release();
        delete h;
        return rc;
    }
    *out = h;
    return PSST_OK;
}

namespace {

int launch_chunks(psst_net *h, long long step0, long long n_steps, long long chunk, cudaStream_t st);

// Launch the kernels for n_steps steps starting at global step `step0`.
int launch_steps(psst_net *h, long long step0, long long n_steps, cudaStream_t st) {
    const long long chunk = 1LL << 30;
    const bool fork = h->mode != PSST_MODE_GRID && !h->class_streams.empty();
    if (fork) {
        // the class streams start after everything queued on st so far
        cudaError_t e = cudaEventRecord(h->class_events[0], st);
        for (size_t c = 0; e == cudaSuccess && c < h->class_streams.size(); ++c)
            e = cudaStreamWaitEvent(h->class_streams[c], h->class_events[0], 0);
        if (e != cudaSuccess) return cuda_fail(e, "psst_integrate fork");
    }
    const int rc = launch_chunks(h, step0, n_steps, chunk, st);
    if (fork) {
        // st continues once every class is done (also on a launch error)
        cudaError_t e = cudaSuccess;
        for (size_t c = 0; c < h->class_streams.size(); ++c) {
            const cudaError_t e1 = cudaEventRecord(h->class_events[1 + c], h->class_streams[c]);
            const cudaError_t e2 = cudaStreamWaitEvent(st, h->class_events[1 + c], 0);
            if (e == cudaSuccess) e = e1 != cudaSuccess ? e1 : e2;
        }
        if (e != cudaSuccess && !rc) return cuda_fail(e, "psst_integrate join");
    }
    return rc;
}

int launch_chunks(psst_net *h, long long step0, long long n_steps, long long chunk, cudaStream_t st) {
    for (long long done = 0; done < n_steps;) {
        const int n = (int)std::min<long long>(chunk, n_steps - done);
        if (h->mode == PSST_MODE_GRID) {
            cudaError_t e = psst::grid_launch(h->v, h->gv, step0 + done, n, h->grid, h->block, h->smem, st);
            if (e != cudaSuccess) return cuda_fail(e, "psst_integrate launch");
            ++h->launches;
        } else {
            const bool fork = !h->class_streams.empty();
            for (size_t c = 0; c < h->classes.size(); ++c) {
                cudaError_t e = psst::cta_launch(h->v, h->classes[c], step0 + done, n,
                                                 fork ? h->class_streams[c] : st);
                if (e != cudaSuccess) return cuda_fail(e, "psst_integrate launch");
                ++h->launches;
            }
            if (h->n_ind_neurons > 0) {
                cudaError_t e = psst::indep_launch(h->v, h->d_ind_neuron, h->d_ind_net, h->n_ind_neurons,
                                                   step0 + done, n, fork ? h->class_streams.back() : st);
                if (e != cudaSuccess) return cuda_fail(e, "psst_integrate launch");
                ++h->launches;
            }
        }
        done += n;
    }
    return PSST_OK;
}

// Kernel nodes take the global step index as an argument: net_kernel's and
// indep_kernel's 4th (v, list, plans | ind_neuron, ind_net, step0, ...),
// grid_kernel's 3rd (v, g, step0, nsteps).  The captured graph keeps each
// node's arguments as captured, so a node's step index minus the step at
// capture is its offset within the call (0, or a multiple of the launch
// chunk when the call spans several chunks); the replay gives it the same
// offset from its own first step, whatever order the nodes are listed in.
int patch_step0(psst_net *h, long long step0) {
    size_t n = 0;
    cudaError_t e = cudaGraphGetNodes(h->graph, nullptr, &n);
    std::vector<cudaGraphNode_t> nodes(n);
    if (e == cudaSuccess && n) e = cudaGraphGetNodes(h->graph, nodes.data(), &n);
    const int idx = h->mode == PSST_MODE_GRID ? 2 : 3;
    const int nargs = h->mode == PSST_MODE_GRID ? 4 : 6;
    for (size_t i = 0; e == cudaSuccess && i < n; ++i) {
        cudaGraphNodeType t;
        e = cudaGraphNodeGetType(nodes[i], &t);
        if (e != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams p;
        e = cudaGraphKernelNodeGetParams(nodes[i], &p);
        if (e != cudaSuccess) break;
        const long long captured = *(const long long *)p.kernelParams[idx];
        long long s = step0 + (captured - h->graph_step0);
        void *args[6];
        for (int q = 0; q < nargs; ++q) args[q] = p.kernelParams[q];
        args[idx] = &s;
        p.kernelParams = args;
        e = cudaGraphExecKernelNodeSetParams(h->graph_exec, nodes[i], &p);
    }
    return e == cudaSuccess ? PSST_OK : cuda_fail(e, "graph update");
}

// Integrate through a CUDA graph of the launch sequence: captured once per
// step count, then replayed with the step index patched into its kernels.
int replay_steps(psst_net *h, long long step0, long long n_steps, cudaStream_t st) {
    if (!h->graph_exec || h->graph_nsteps != n_steps) {
        h->drop_graph();
        cudaStream_t cs;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e, "graph stream");
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        int rc = PSST_OK;
        if (e == cudaSuccess) rc = launch_steps(h, step0, n_steps, cs);
        cudaGraph_t g = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&h->graph_exec, g, 0);
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(e, "graph capture");
        }
        h->graph = g;
        h->graph_nsteps = n_steps;
        h->graph_step0 = step0;
        h->graph_launches = h->launches;
    } else {
        const int rc = patch_step0(h, step0);
        if (rc) return rc;
    }
    h->launches = h->graph_launches;
    const cudaError_t e = cudaGraphLaunch(h->graph_exec, st);
    return e == cudaSuccess ? PSST_OK : cuda_fail(e, "graph launch");
}

// After the state was replaced: which networks now have equal gates within
// every (presynaptic neuron, type) pair?  When that changes, the CTA-mode
// plan (per-pair or per-synapse layout) is rebuilt.
int recheck_pairs(psst_net *h, cudaStream_t st) {
    if (h->pin.force_synapse_gates) return PSST_OK;
    const int n_nets = h->pin.n_nets;
    if (!h->d_check) {
        cudaError_t e = h->alloc(&h->d_check, (size_t)n_nets);
        if (e != cudaSuccess) return cuda_fail(e, "pair check buffer");
    }
    int max_m = 0;
    for (int b = 0; b < n_nets; ++b) max_m = std::max(max_m, (h->pin.net_off[b + 1] - h->pin.net_off[b]) * h->pin.nt);
    std::vector<uint8_t> ok((size_t)n_nets, 0);
    if (4LL * max_m <= 200 * 1024) {
        cudaError_t e = psst::pair_check(h->v, h->d_check, 4 * max_m, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(ok.data(), h->d_check, (size_t)n_nets, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_fail(e, "pair check");
    }
    bool changed = false;
    for (int b = 0; b < n_nets; ++b) {
        const uint8_t f = (uint8_t)((h->pin.flags[b] & psst::NET_HAS2) | (ok[b] ? psst::NET_PAIR : 0));
        changed |= f != h->pin.flags[b];
        h->pin.flags[b] = f;
    }
    if (!changed) return PSST_OK;
    cudaError_t e = cudaMemcpy((void *)h->v.net_flags, h->pin.flags.data(), (size_t)n_nets, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "flags");
    h->drop_graph();
    return h->mode == PSST_MODE_GRID ? setup_grid(h, h->caps, &e) : setup_cta(h, h->caps, &e);
}

}  // namespace

int psst_set_graph_mode(psst_net *h, int enable) {
    if (!h) return fail(PSST_ERR_INVALID_ARG, "handle is NULL");
    DeviceGuard guard(h->device);
    h->graph_mode = enable != 0;
    if (!enable) h->drop_graph();
    return PSST_OK;
}

int psst_autotune(psst_net *h, int64_t trial_steps, void *stream) {
    if (!h) return fail(PSST_ERR_INVALID_ARG, "handle is NULL");
    if (trial_steps < 1) return fail(PSST_ERR_INVALID_ARG, "trial_steps must be >= 1");
    if (h->mode != PSST_MODE_CTA) return PSST_OK;  // grid mode has one shape per device
    DeviceGuard guard(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const size_t dim = (size_t)(4 * h->v.N + 2 * h->v.S);
    cudaError_t e = cudaSuccess;
    // the state and its remainders, restored after the trials
    if (!h->tune_buf) e = h->alloc(&h->tune_buf, 2 * dim);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->tune_buf, h->v.state, dim * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->tune_buf + dim, h->v.state_lo, dim * sizeof(float), cudaMemcpyDeviceToDevice, st);
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&ev1);
    // the record ring may be written by trial steps: trials run with recording off
    const int stride = h->v.rec_stride;
    h->v.rec_stride = 0;
    // few CTAs for the GPU: try spreading each network over a cluster of 2 or 4
    int sms = 0;
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e == cudaSuccess && h->pin.tune_cl && 2LL * h->grid <= sms && !h->classes.empty()) {
        const int n = (int)std::min<long long>(trial_steps, 1 << 20);
        float best = 1e30f;
        int best_cl = h->pin.min_cl;
        for (int mc = 1; mc <= PSST_MAX_CL && e == cudaSuccess; mc *= 2) {
            h->pin.min_cl = mc;
            if (setup_cta(h, h->caps, &e) != PSST_OK) {
                e = cudaSuccess;
                continue;
            }
            float ms = 0.0f;
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // warm-up, then timed
                e = cudaMemcpyAsync(h->v.state, h->tune_buf, dim * sizeof(float), cudaMemcpyDeviceToDevice, st);
                if (e == cudaSuccess) e = cudaEventRecord(ev0, st);
                if (e == cudaSuccess && launch_steps(h, 0, n, st) != PSST_OK) e = cudaErrorUnknown;
                if (e == cudaSuccess) e = cudaEventRecord(ev1, st);
                if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
            }
            if (e == cudaSuccess && ms < best) {
                best = ms;
                best_cl = mc;
            }
        }
        h->pin.min_cl = best_cl;
        if (e == cudaSuccess && setup_cta(h, h->caps, &e) != PSST_OK && e == cudaSuccess) e = cudaErrorUnknown;
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->v.state, h->tune_buf, dim * sizeof(float), cudaMemcpyDeviceToDevice, st);
    }
    for (size_t ci = 0; e == cudaSuccess && ci < h->classes.size(); ++ci) {
        psst::ClassLaunch &c = h->classes[ci];
        // the class's CTAs per SM are fixed by its shared memory and its
        // default CTA keeps 1024 threads per SM (64 registers each); the
        // trials try twice, once, half and a quarter of that size, each with
        // the planned copies of the per-pair gate table and with one copy
        const int base = c.block;
        float best = 1e30f;
        int best_block = base, best_cap = c.lrep_cap;
        for (int trial = 0; trial < 8; ++trial) {
            const int b = trial / 2 == 0 ? 2 * base : base >> (trial / 2 - 1);
            const int cap = trial % 2 ? 0 : c.lrep_cap;
            if (b > 1024 || b < 64 || b % 32 || (trial % 2 && c.lrep_cap == 0)) continue;
            psst::ClassLaunch t = c;
            t.block = b;
            t.lrep_cap = cap;
            const int n = (int)std::min<long long>(trial_steps, 1 << 20);
            e = psst::cta_launch(h->v, t, 0, n, st);  // warm-up
            if (e != cudaSuccess) {
                cudaGetLastError();  // a shape that cannot launch is skipped
                e = cudaSuccess;
                continue;
            }
            cudaEventRecord(ev0, st);
            e = psst::cta_launch(h->v, t, 0, n, st);
            cudaEventRecord(ev1, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev0, ev1);
            if (e == cudaSuccess && ms < best) {
                best = ms;
                best_block = b;
                best_cap = cap;
            }
        }
        c.block = best_block;
        c.lrep_cap = best_cap;
    }
    h->v.rec_stride = stride;
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->v.state, h->tune_buf, dim * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(h->v.state_lo, h->tune_buf + dim, dim * sizeof(float), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (ev0) cudaEventDestroy(ev0);
    if (ev1) cudaEventDestroy(ev1);
    h->drop_graph();
    if (!h->classes.empty()) h->block = h->classes.back().block;
    return e == cudaSuccess ? PSST_OK : cuda_fail(e, "psst_autotune");
}

// PSST_SYNC set to anything but "0": psst_integrate waits for its work and
// reports device-side failures itself (debugging aid).
static bool sync_requested() {
    const char *s = std::getenv("PSST_SYNC");
    return s && *s && std::strcmp(s, "0") != 0;
}

static int integrate_async(psst_net *h, int64_t n_steps, cudaStream_t st);

int psst_integrate(psst_net *h, int64_t n_steps, void *stream) {
    const int rc = integrate_async(h, n_steps, (cudaStream_t)stream);
    if (rc || !h || !sync_requested()) return rc;
    return psst_status(h, stream);
}

static int integrate_async(psst_net *h, int64_t n_steps, cudaStream_t stream) {
    if (!h) return fail(PSST_ERR_INVALID_ARG, "handle is NULL");
    if (n_steps < 0) return fail(PSST_ERR_INVALID_ARG, "n_steps must be >= 0");
    h->launches = 0;
    if (n_steps == 0) return PSST_OK;
    DeviceGuard guard(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    if (h->rec_ck_every <= 0) {
        const int rc = h->graph_mode ? replay_steps(h, h->step, n_steps, st) : launch_steps(h, h->step, n_steps, st);
        if (rc) return rc;
        h->step += n_steps;
        return PSST_OK;
    }
    // recording checkpoints: the state at the start and after every rec_ck_every steps
    if (n_steps > h->rec_ck_cap_steps)
        return fail(PSST_ERR_INVALID_ARG, "n_steps %lld exceeds the checkpoint capacity %lld", (long long)n_steps,
                    h->rec_ck_cap_steps);
    const size_t dim = (size_t)(4 * h->v.N + 2 * h->v.S);
    h->rec_ck_valid = false;
    const long long s0 = h->step;
    for (long long done = 0, c = 0; done < n_steps; ++c) {
        cudaError_t e = cudaMemcpyAsync(h->rec_ck + c * dim, h->v.state, dim * sizeof(float),
                                        cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->rec_ck_lo + c * dim, h->v.state_lo, dim * sizeof(float), cudaMemcpyDeviceToDevice,
                                st);
        if (e != cudaSuccess) return cuda_fail(e, "checkpoint copy");
        const long long n = std::min<long long>(h->rec_ck_every, n_steps - done);
        const int rc = launch_steps(h, s0 + done, n, st);
        if (rc) return rc;
        done += n;
    }
    h->step += n_steps;
    h->rec_ck_start = s0;
    h->rec_ck_nsteps = n_steps;
    h->rec_ck_spacing = h->rec_ck_every;
    h->rec_ck_valid = true;
    return PSST_OK;
}

int psst_record_checkpoints(psst_net *h, int32_t every, int64_t max_steps) {
    if (!h) return fail(PSST_ERR_INVALID_ARG, "handle is NULL");
    if (every < 0 || (every > 0 && max_steps < 1)) return fail(PSST_ERR_INVALID_ARG, "bad checkpoint spacing");
    if (h->mode != PSST_MODE_CTA && every > 0) return fail(PSST_ERR_UNSUPPORTED, "checkpoints need CTA mode");
    h->rec_ck_valid = false;
    h->rec_ck_every = every;
    if (every == 0) return PSST_OK;
    // the buffers hold whole checkpoints: a call of max_steps steps records
    // ceil(max_steps / every) of them
    const long long dim = 4 * h->v.N + 2 * h->v.S;
    const long long need = ((max_steps + every - 1) / every) * dim;
    if (need > h->rec_ck_cap || !h->rec_ck) {
        DeviceGuard guard(h->device);
        cudaError_t e = h->alloc(&h->rec_ck, (size_t)need);
        if (e == cudaSuccess) e = h->alloc(&h->rec_ck_lo, (size_t)need);
        if (e != cudaSuccess) {
            h->rec_ck = h->rec_ck_lo = nullptr;
            h->rec_ck_cap = 0;
            h->rec_ck_cap_steps = 0;
            h->rec_ck_every = 0;
            return cuda_fail(e, "checkpoint buffer");
        }
        h->rec_ck_cap = need;
    }
    // the steps one integrate call may record at this spacing
    h->rec_ck_cap_steps = (h->rec_ck_cap / dim) * every;
    return PSST_OK;
}

int psst_set_barrier_timeout(psst_net *h, int64_t timeout_ns) {
    if (!h) return fail(PSST_ERR_INVALID_ARG, "handle is NULL");
    if (timeout_ns < 0) return fail(PSST_ERR_INVALID_ARG, "timeout must be >= 0");
    h->gv.timeout_ns = (unsigned long long)timeout_ns;
    return PSST_OK;
}

int psst_status(psst_net *h, void *stream) {
    if (!h) return fail(PSST_ERR_INVALID_ARG, "handle is NULL");
    DeviceGuard guard(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    int code = 0;
    cudaError_t e = cudaMemcpyAsync(&code, h->v.err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->v.err, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_fail(e, "psst_status");
    if (code) return fail(code, "device reported: %s", psst_error_string(code));
    return PSST_OK;
}

int psst_get_state(const psst_net *h, float *dst, size_t n, int dst_on_device, void *stream) {
    if (!h || !dst) return fail(PSST_ERR_INVALID_ARG, "NULL argument");
    const size_t dim = (size_t)(4 * h->v.N + 2 * h->v.S);
    if (n < dim) return fail(PSST_ERR_INVALID_ARG, "dst holds %zu floats, state has %zu", n, dim);
    DeviceGuard guard(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(dst, h->v.state, dim * sizeof(float),
                                    dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && !dst_on_device) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? PSST_OK : cuda_fail(e, "psst_get_state");
}

int psst_set_state(psst_net *h, const float *src, size_t n, int src_on_device, void *stream) {
    if (h) h->rec_ck_valid = false;
    if (!h || !src) return fail(PSST_ERR_INVALID_ARG, "NULL argument");
    const size_t dim = (size_t)(4 * h->v.N + 2 * h->v.S);
    if (n != dim) return fail(PSST_ERR_INVALID_ARG, "src holds %zu floats, state has %zu", n, dim);
    DeviceGuard guard(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(h->v.state, src, dim * sizeof(float),
                                    src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    // an FP32 state given by the caller is exact: its remainders are zero
    if (e == cudaSuccess) e = cudaMemsetAsync(h->v.state_lo, 0, dim * sizeof(float), st);
    if (e == cudaSuccess && !src_on_device) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "psst_set_state");
    return recheck_pairs(h, st);
}

int psst_set_step(psst_net *h, int64_t step) {
    if (!h) return fail(PSST_ERR_INVALID_ARG, "handle is NULL");
    if (step < 0) return fail(PSST_ERR_INVALID_ARG, "step must be >= 0");
    h->step = step;
    h->rec_reset = step;
    h->rec_ck_valid = false;
    return PSST_OK;
}

int psst_read_record(const psst_net *h, float *dst, size_t cap_frames, int64_t *n_frames, int dst_on_device,
                     void *stream) {
    if (!h || !n_frames) return fail(PSST_ERR_INVALID_ARG, "NULL argument");
    *n_frames = 0;
    if (h->v.rec_stride <= 0) return PSST_OK;
    const long long stride = h->v.rec_stride, cap = h->v.rec_cap, N = h->v.N;
    const long long f_end = h->step / stride;        // frames 0..f_end-1 exist up to now
    const long long f_begin0 = h->rec_reset / stride;  // first frame since the last reset
    long long count = std::max(0LL, f_end - f_begin0);
    count = std::min(count, cap);
    count = std::min<long long>(count, (long long)cap_frames);
    if (count == 0) return PSST_OK;
    if (!dst) return fail(PSST_ERR_INVALID_ARG, "dst is NULL");
    DeviceGuard guard(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    long long f = f_end - count;
    long long written = 0;
    cudaError_t e = cudaSuccess;
    while (written < count && e == cudaSuccess) {
        const long long slot = f % cap;
        const long long run = std::min(count - written, cap - slot);
        e = cudaMemcpyAsync(dst + written * N, h->v.rec + slot * N, (size_t)(run * N) * sizeof(float), kind, st);
        written += run;
        f += run;
    }
    if (e == cudaSuccess && !dst_on_device) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(e, "psst_read_record");
    *n_frames = count;
    return PSST_OK;
}

int psst_set_weights(psst_net *h, const float *w, size_t n, int on_device, void *stream) {
    if (h) h->rec_ck_valid = false;
    if (!h || !w) return fail(PSST_ERR_INVALID_ARG, "NULL argument");
    if (n != (size_t)h->v.S) return fail(PSST_ERR_INVALID_ARG, "weights hold %zu values, network has %lld", n, h->v.S);
    DeviceGuard guard(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync((void *)h->v.weight, w, n * sizeof(float),
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? PSST_OK : cuda_fail(e, "psst_set_weights");
}

int psst_set_neuron_params(psst_net *h, const float *p, size_t n, int on_device, void *stream) {
    if (h) h->rec_ck_valid = false;
    if (!h || !p) return fail(PSST_ERR_INVALID_ARG, "NULL argument");
    if (n != (size_t)h->n_ntypes * PSST_NEURON_NPARAM)
        return fail(PSST_ERR_INVALID_ARG, "parameter table holds %zu values, expected %d", n,
                    h->n_ntypes * PSST_NEURON_NPARAM);
    DeviceGuard guard(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync((void *)h->v.nparams, p, n * sizeof(float),
                                    on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !on_device) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? PSST_OK : cuda_fail(e, "psst_set_neuron_params");
}

int psst_adjoint(psst_net *h, int64_t n_steps, const float *dL_dV, int64_t n_frames, int32_t ckpt_every,
                 float *grad_w, float *grad_neuron_params, float *grad_state0, void *stream) {
    if (!h || !grad_w || !grad_neuron_params) return fail(PSST_ERR_INVALID_ARG, "NULL argument");
    if (h->mode != PSST_MODE_CTA) return fail(PSST_ERR_UNSUPPORTED, "the adjoint runs in CTA mode only");
    if (n_steps < 1 || n_steps > (1LL << 30)) return fail(PSST_ERR_INVALID_ARG, "n_steps must be in 1..2^30");
    if (ckpt_every == 0) {
        if (!h->rec_ck_valid || h->rec_ck_nsteps != n_steps)
            return fail(PSST_ERR_STATE, "no checkpoints of a %lld-step integrate call are recorded", (long long)n_steps);
    } else if (ckpt_every < 1) {
        return fail(PSST_ERR_INVALID_ARG, "ckpt_every must be >= 1 (0 = recorded)");
    }
    const long long stride = h->v.rec_stride, s0 = ckpt_every == 0 ? h->rec_ck_start : h->step;
    long long want = 0;
    if (stride > 0) want = (s0 + n_steps) / stride - s0 / stride;
    if (n_frames != want)
        return fail(PSST_ERR_INVALID_ARG, "dL_dV has %lld frames, the span records %lld", (long long)n_frames, want);
    if (n_frames > 0 && !dL_dV) return fail(PSST_ERR_INVALID_ARG, "dL_dV is NULL");
    DeviceGuard guard(h->device);
    const int n_nets = h->v.n_nets, nt = h->v.n_stypes;
    cudaError_t e = cudaSuccess;
    if (ckpt_every > 0) {
        // The span's checkpoints: the forward kernel integrates it once from
        // the current state, recording the state and its remainders every
        // ckpt_every steps, so that each segment the adjoint recomputes
        // starts on the forward kernel's trajectory; the network's state,
        // step, record ring and recording setting are then put back.
        const size_t dim = (size_t)(4 * h->v.N + 2 * h->v.S);
        cudaStream_t st = (cudaStream_t)stream;
        if (!h->tune_buf) e = h->alloc(&h->tune_buf, 2 * dim);
        if (e == cudaSuccess) e = cudaMemcpyAsync(h->tune_buf, h->v.state, dim * sizeof(float), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->tune_buf + dim, h->v.state_lo, dim * sizeof(float), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_fail(e, "psst_adjoint state copy");
        const int keep_every = h->rec_ck_every, keep_stride = h->v.rec_stride;
        const long long keep_step = h->step;
        h->v.rec_stride = 0;
        int rc = psst_record_checkpoints(h, ckpt_every, n_steps);
        if (rc == PSST_OK) rc = integrate_async(h, n_steps, st);
        h->v.rec_stride = keep_stride;
        h->rec_ck_every = keep_every;
        h->rec_ck_cap_steps = keep_every > 0 ? (h->rec_ck_cap / (long long)dim) * keep_every : 0;
        h->step = keep_step;
        e = cudaMemcpyAsync(h->v.state, h->tune_buf, dim * sizeof(float), cudaMemcpyDeviceToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->v.state_lo, h->tune_buf + dim, dim * sizeof(float), cudaMemcpyDeviceToDevice, st);
        if (rc != PSST_OK) return rc;
        if (e != cudaSuccess) return cuda_fail(e, "psst_adjoint state copy");
    }
    ckpt_every = h->rec_ck_spacing;
    // per-network plan (host copy of the CSR offsets is not kept: read them back once)
    if (h->adj_K.empty()) {
        std::vector<int> off((size_t)n_nets + 1);
        std::vector<long long> rp((size_t)h->v.N + 1);
        e = cudaMemcpy(off.data(), h->v.net_off, off.size() * sizeof(int), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(rp.data(), h->v.row_ptr, rp.size() * sizeof(long long), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "psst_adjoint plan");
        std::vector<uint32_t> code((size_t)h->v.S);
        e = cudaMemcpy(code.data(), h->v.syn_code, code.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "psst_adjoint plan");
        h->adj_K.resize(n_nets);
        h->adj_items.resize(n_nets);
        std::vector<int> KC((size_t)n_nets), citems((size_t)n_nets), cib, ck;
        std::vector<unsigned short> crow;
        std::vector<long long> cslot_off((size_t)n_nets), cib_off((size_t)n_nets);
        long long slots = 0;
        int need = 0;
        for (int b = 0; b < n_nets; ++b) {
            const int n0 = off[b], N = off[b + 1] - n0, M = N * nt;
            const long long S = rp[n0 + N] - rp[n0], sb = rp[n0];
            // row items (forward CTA): chunks per item a power of two (1..8),
            // about 1024 items per network
            const int K0 = (int)std::max(1LL, std::min(8LL, (S / 4 + 1023) / 1024));
            const int K = K0 >= 8 ? 8 : K0 >= 4 ? 4 : K0 >= 2 ? 2 : 1;
            int items = 0;
            for (int i = n0; i < n0 + N; ++i) items += (int)((rp[i + 1] - rp[i] + 4 * K - 1) / (4 * K));
            // inert items after the rows' make the chunk-plane stride congruent to
            // 8/K modulo 8 (K = 8: odd), so that the 8 groups of 4 lanes reading
            // consecutive synapses of a row (over planes j < K and items q < 8/K)
            // start on 8 different 4-bank groups
            while (items % 8 != (8 / K) % 8 && !(K == 8 && items % 2 == 1)) ++items;
            if (N >= 65536 || (long long)M >= 65536)
                return fail(PSST_ERR_UNSUPPORTED, "adjoint: net %d too large (%d neurons)", b, N);
            // column items (sweeping CTA): the smallest chunks per item (1..8)
            // that leave at most one item per thread, each pair's synapses
            // dealt round-robin over its items (rows in CSR order)
            std::vector<int> cnt((size_t)M, 0);
            for (long long k = sb; k < sb + S; ++k) ++cnt[code[(size_t)k] & 0xFFFFFFu];
            int kc = 1, nci = 0;
            for (;; kc *= 2) {
                nci = 0;
                for (int q = 0; q < M; ++q) nci += (cnt[q] + 4 * kc - 1) / (4 * kc);
                if (nci <= 1024 || kc == 8) break;
            }
            const long long bytes = psst::adj_smem_need(N, nt, items, K, nci, kc);
            if (bytes > h->max_dyn)
                return fail(PSST_ERR_UNSUPPORTED, "adjoint: net %d needs %lld B of shared memory (max %d)", b, bytes,
                            h->max_dyn);
            need = std::max<int>(need, (int)bytes);
            cib_off[b] = (long long)cib.size();
            std::vector<int> first((size_t)M + 1), seen((size_t)M, 0);
            int acc = 0;
            for (int q = 0; q < M; ++q) {
                first[q] = acc;
                acc += (cnt[q] + 4 * kc - 1) / (4 * kc);
            }
            first[M] = acc;
            cib.insert(cib.end(), first.begin(), first.end());
            cslot_off[b] = slots;
            const long long cslots = 4LL * kc * nci;
            ck.resize((size_t)(slots + cslots), -1);
            crow.resize((size_t)(slots + cslots), 0);
            for (int i = n0; i < n0 + N; ++i)
                for (long long k = rp[i]; k < rp[i + 1]; ++k) {
                    const int q = (int)(code[(size_t)k] & 0xFFFFFFu), nq = first[q + 1] - first[q];
                    const int m = seen[q]++, t = first[q] + m % nq, pos = m / nq;
                    const long long slot = slots + ((long long)(pos >> 2) * nci + t) * 4 + (pos & 3);
                    ck[(size_t)slot] = (int)(k - sb);
                    crow[(size_t)slot] = (unsigned short)(i - n0);
                }
            h->adj_K[b] = K;
            h->adj_items[b] = items;
            KC[b] = kc;
            citems[b] = nci;
            slots += cslots;
        }
        h->adj_smem = need;
        e = upload(h, &h->d_adjK, h->adj_K.data(), h->adj_K.size());
        if (e == cudaSuccess) e = upload(h, &h->d_adjI, h->adj_items.data(), h->adj_items.size());
        if (e == cudaSuccess) e = upload(h, &h->d_adjKC, KC.data(), KC.size());
        if (e == cudaSuccess) e = upload(h, &h->d_adjCI, citems.data(), citems.size());
        if (e == cudaSuccess) e = upload(h, &h->d_cib, cib.data(), cib.size());
        if (e == cudaSuccess) e = upload(h, &h->d_ciboff, cib_off.data(), cib_off.size());
        if (e == cudaSuccess) e = upload(h, &h->d_ck, ck.data(), ck.size());
        if (e == cudaSuccess) e = upload(h, &h->d_crow, crow.data(), crow.size());
        if (e == cudaSuccess) e = upload(h, &h->d_cslotoff, cslot_off.data(), cslot_off.size());
        if (e == cudaSuccess) e = h->alloc(&h->adj_gpart, (size_t)slots / 4);
        if (e == cudaSuccess) e = h->alloc(&h->adj_gtot, (size_t)slots);
        if (e == cudaSuccess) e = h->alloc(&h->adj_gpn, (size_t)h->v.N * 9);
        if (e == cudaSuccess) e = h->alloc(&h->adj_gy0, (size_t)h->v.N * 4);
        if (e == cudaSuccess) e = h->alloc(&h->d_segoff, (size_t)n_nets);
        if (e != cudaSuccess) return cuda_fail(e, "psst_adjoint buffers");
    }
    // checkpoint and segment storage for this span (grown on demand)
    {
        std::vector<int> off((size_t)n_nets + 1);
        e = cudaMemcpy(off.data(), h->v.net_off, off.size() * sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "psst_adjoint offsets");
        std::vector<long long> sg((size_t)n_nets);
        long long seg_total = 0;
        for (int b = 0; b < n_nets; ++b) {
            const long long N = off[b + 1] - off[b];
            const long long step_floats = psst::adj_segment_floats(h->v.method, h->v.rk_ns, (int)N, nt);  // one step's stages
            sg[b] = seg_total;
            seg_total += 2LL * std::min<long long>(ckpt_every, n_steps) * step_floats;  // two buffers
        }
        if (seg_total > h->adj_seg_cap) {
            e = h->alloc(&h->adj_seg, (size_t)seg_total);
            h->adj_seg_cap = seg_total;
        }
        if (e == cudaSuccess) e = cudaMemcpy(h->d_segoff, sg.data(), sg.size() * sizeof(long long), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "psst_adjoint storage");
    }
    psst::AdjView av{};
    av.K = h->d_adjK;
    av.n_items = h->d_adjI;
    av.KC = h->d_adjKC;
    av.n_citems = h->d_adjCI;
    av.cib = h->d_cib;
    av.cib_off = h->d_ciboff;
    av.ck = h->d_ck;
    av.crow = h->d_crow;
    av.cslot_off = h->d_cslotoff;
    av.ckpt_every = ckpt_every;
    av.ck_full = h->rec_ck;
    av.ck_full_lo = h->rec_ck_lo;
    av.dim = 4 * h->v.N + 2 * h->v.S;
    av.seg = h->adj_seg;
    av.seg_off = h->d_segoff;
    av.gpart = h->adj_gpart;
    av.gtot = h->adj_gtot;
    av.dLdV = dL_dV;
    av.n_frames = (int)n_frames;
    av.grad_w = grad_w;
    av.gp_neuron = h->adj_gpn;
    av.grad_y0 = grad_state0 ? grad_state0 : h->adj_gy0;
    e = psst::adj_launch(h->v, av, s0, (int)n_steps, h->adj_smem, h->n_ntypes, grad_neuron_params,
                         (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "psst_adjoint launch");
    h->launches = 2;
    return PSST_OK;
}

int psst_query(const psst_net *h, psst_info *out) {
    if (!h || !out) return fail(PSST_ERR_INVALID_ARG, "NULL argument");
    std::memset(out, 0, sizeof *out);
    out->n_nets = h->v.n_nets;
    out->n_neurons = h->v.N;
    out->n_synapses = h->v.S;
    out->steps_done = h->step;
    out->rec_frames = h->v.rec_stride > 0 ? h->step / h->v.rec_stride - h->rec_reset / h->v.rec_stride : 0;
    out->mode = h->mode;
    out->block_threads = h->block;
    out->item_chunks = h->K;
    out->grid_ctas = h->grid;
    out->smem_bytes = h->smem;
    out->n_single_cta_nets = h->n_smem;
    out->n_cluster_nets = h->n_global;
    out->n_launch_classes = (int32_t)h->classes.size();
    out->kernel_launches = h->launches;
    out->n_independent_nets = h->mode == PSST_MODE_GRID ? 0 : h->n_ind_nets;
    if (h->mode == PSST_MODE_GRID) {
        out->n_pair_gate_nets = h->gv.pair;
    } else {
        for (uint8_t f : h->pin.flags) out->n_pair_gate_nets += (f & psst::NET_PAIR) ? 1 : 0;
    }
    out->ck_start = h->rec_ck_valid ? h->rec_ck_start : -1;
    out->ck_steps = h->rec_ck_valid ? h->rec_ck_nsteps : 0;
    return PSST_OK;
}

int psst_destroy_network(psst_net *h) {
    if (!h) return PSST_OK;
    {
        DeviceGuard guard(h->device);
        cudaDeviceSynchronize();
        h->release();
    }
    delete h;
    return PSST_OK;
}

}  // extern "C"
