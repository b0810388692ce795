// C interface (include/psst.h): validation, device layout, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <cmath>
#include <cstdarg>
#include <cstdio>
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

struct psst_net {
    int device = 0;
    NetView v{};
    psst::GridView gv{};
    std::vector<psst::ClassLaunch> classes;  // CTA mode: one launch per size class
    std::vector<void *> allocs;
    long long step = 0;       // global step index of the current state
    long long rec_reset = 0;  // step at which the record ring was last reset
    int mode = PSST_MODE_CTA;
    int block = 0, G = 0, smem = 0, grid = 0;
    int n_smem = 0, n_global = 0;
    int launches = 0;

    template <class T>
    cudaError_t alloc(T **p, size_t count) {
        void *q = nullptr;
        cudaError_t e = cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T));
        if (e == cudaSuccess) allocs.push_back(q);
        *p = (T *)q;
        return e;
    }
    void release() {
        for (void *p : allocs) cudaFree(p);
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
    if (d->row_group && (d->row_group > 32 || (d->row_group & (d->row_group - 1))))
        return fail(PSST_ERR_INVALID_ARG, "row_group must be a power of two <= 32");
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
    return PSST_OK;
}

// Per-row chunk counts (first- and second-order parts padded to 4) of the
// whole batch, and which networks hold second-order synapses.
void row_chunk_counts(const psst_network_desc *d, std::vector<int> &rowch, std::vector<uint8_t> &has2) {
    const long long N = d->net_neuron_off[d->n_nets];
    rowch.assign((size_t)N, 0);
    has2.assign((size_t)d->n_nets, 0);
    for (int b = 0; b < d->n_nets; ++b) {
        for (long long i = d->net_neuron_off[b]; i < d->net_neuron_off[b + 1]; ++i) {
            int n1 = 0, n2 = 0;
            for (long long k = d->row_ptr[i]; k < d->row_ptr[i + 1]; ++k) {
                if (d->syn_params[(size_t)d->syn_type[k] * PSST_SYN_NPARAM] != 0.0f) ++n2;
                else ++n1;
            }
            rowch[i] = psst::row_chunks(n1, n2);
            if (n2) has2[b] = 1;
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

// Shared memory of one CTA owning rows [r0, r1) of an N-neuron network
// (CTA/cluster mode: the neuron part covers all N neurons).
long long cta_need(int N, int nt, bool has2, const int *rowch, int r0, int r1) {
    long long ch = 0;
    for (int i = r0; i < r1; ++i) ch += rowch[i];
    const psst::NeuronLayout L = psst::make_nlayout(N, nt, has2, r1 - r0);
    return L.syn + psst::syn_smem_bytes(ch, r1 - r0, has2);
}

// Lanes per CSR row: the power of two nearest half the mean number of
// chunks per row, clamped to 2..32.
int default_row_group(double mean_chunks) {
    int g = 2;
    while (g < 32 && g < mean_chunks * 0.5) g <<= 1;
    return g;
}

// Grid mode: one contiguous block of rows per CTA with balanced cost
// (chunks plus a per-neuron share); the double-buffered gate-map tables and
// the barrier words.
int setup_grid(psst_net *h, const psst_network_desc *d, int max_smem, bool has2, const std::vector<int> &rowch,
               cudaError_t *err) {
    const long long N = h->v.N;
    const int nt = h->v.n_stypes;
    if (N * nt >= 65536)
        return fail(PSST_ERR_UNSUPPORTED, "grid mode: %lld neurons x %d synapse types must stay below 65536", N, nt);
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device);
    if (e != cudaSuccess) return *err = e, cuda_fail(e, "device attributes");
    const int parts = (int)std::max<long long>(1, std::min<long long>(sms, (N + 7) / 8));
    std::vector<double> cost((size_t)N);
    for (long long i = 0; i < N; ++i) cost[i] = rowch[i] + 10.0;
    std::vector<int> split;
    balanced_split(cost, parts, split);
    std::vector<int> chunks((size_t)parts, 0);
    int need = 0;
    for (int c = 0; c < parts; ++c) {
        const int n = split[c + 1] - split[c];
        long long ch = 0;
        for (int i = split[c]; i < split[c + 1]; ++i) ch += rowch[i];
        const long long bytes = psst::make_nlayout(n, nt, has2, n).syn + psst::syn_smem_bytes(ch, n, has2);
        if (bytes > max_smem)
            return fail(PSST_ERR_UNSUPPORTED, "grid mode: block %d needs %lld B of shared memory (max %d)", c, bytes,
                        max_smem);
        chunks[c] = (int)ch;
        need = std::max<int>(need, (int)bytes);
    }
    if (!h->block) h->block = 1024;
    if (!h->G) h->G = default_row_group((double)std::accumulate(rowch.begin(), rowch.end(), 0LL) / (double)N);
    h->smem = need;
    int per_sm = 0;
    e = psst::grid_occupancy(h->block, need, &per_sm);
    if (e != cudaSuccess) return *err = e, cuda_fail(e, "grid occupancy");
    if (per_sm < 1) return fail(PSST_ERR_UNSUPPORTED, "grid mode: a CTA of %d threads does not fit an SM", h->block);
    h->grid = parts;
    h->n_smem = 1;
    psst::GridView &g = h->gv;
    int *rs = nullptr, *chd = nullptr;
    e = upload(h, &rs, split.data(), split.size());
    if (e == cudaSuccess) e = upload(h, &chd, chunks.data(), chunks.size());
    if (e == cudaSuccess) e = h->alloc(&g.c1, (size_t)(2 * N * nt));
    if (e == cudaSuccess && has2) e = h->alloc(&g.c2, (size_t)(2 * N * nt));
    if (e == cudaSuccess) e = h->alloc(&g.bar, 2);
    g.row_split = rs;
    g.chunks = chd;
    g.timeout_ns = 2000000000ULL;
    if (e != cudaSuccess) return *err = e, cuda_fail(e, "grid buffers");
    return PSST_OK;
}

// CTA mode: choose each network's cluster size, group networks into size
// classes (cluster size x CTAs per SM) and upload the launch lists.
int setup_cta(psst_net *h, const psst_network_desc *d, int max_smem, const std::vector<int> &rowch,
              const std::vector<uint8_t> &has2, cudaError_t *err) {
    const int n_nets = d->n_nets, nt = d->n_syn_types;
    std::vector<psst::NetPlan> plans((size_t)n_nets);
    struct Key {
        int cl, tier;
    };
    std::vector<Key> key((size_t)n_nets);
    std::vector<long long> need((size_t)n_nets);
    std::vector<double> cost((size_t)n_nets);
    for (int b = 0; b < n_nets; ++b) {
        const int n0 = d->net_neuron_off[b], N = d->net_neuron_off[b + 1] - n0;
        if ((long long)N * nt >= 65536)
            return fail(PSST_ERR_UNSUPPORTED, "net %d: %d neurons x %d synapse types must stay below 65536", b, N, nt);
        const int *rc = rowch.data() + n0;
        psst::NetPlan &pl = plans[b];
        std::memset(&pl, 0, sizeof pl);
        int chosen = 0;
        long long nd = 0;
        for (int cl = 1; cl <= PSST_MAX_CL && !chosen; cl *= 2) {
            if (cl > 1 && N < 2 * cl) break;
            std::vector<double> c((size_t)N);
            for (int i = 0; i < N; ++i) c[i] = rc[i];
            std::vector<int> split;
            balanced_split(c, cl, split);
            long long worst = 0;
            for (int q = 0; q < cl; ++q) worst = std::max(worst, cta_need(N, nt, has2[b], rc, split[q], split[q + 1]));
            if (worst <= max_smem) {
                chosen = cl;
                nd = worst;
                for (int q = 0; q <= cl; ++q) pl.split[q] = split[q];
                for (int q = 0; q < cl; ++q) {
                    long long ch = 0;
                    for (int i = split[q]; i < split[q + 1]; ++i) ch += rc[i];
                    pl.chunks[q] = (int)ch;
                }
            }
        }
        if (!chosen)
            return fail(PSST_ERR_UNSUPPORTED, "net %d (%d neurons, %lld synapses) does not fit %d CTAs", b, N,
                        (long long)(d->row_ptr[n0 + N] - d->row_ptr[n0]), PSST_MAX_CL);
        const int tier = nd * 4 <= max_smem ? 4 : nd * 2 <= max_smem ? 2 : 1;
        key[b] = {chosen, tier};
        need[b] = nd;
        long long ch = 0;
        for (int i = 0; i < N; ++i) ch += rc[i];
        cost[b] = 4.0 * ch + 30.0 * N;
    }
    // classes in a fixed order: largest networks' classes first
    const int cls[][2] = {{4, 1}, {4, 2}, {4, 4}, {2, 1}, {2, 2}, {2, 4}, {1, 1}, {1, 2}, {1, 4}};
    std::vector<int> all_lists;
    std::vector<std::pair<int, int>> ranges;
    for (auto &ct : cls) {
        std::vector<int> list;
        for (int b = 0; b < n_nets; ++b)
            if (key[b].cl == ct[0] && key[b].tier == ct[1]) list.push_back(b);
        if (list.empty()) continue;
        std::stable_sort(list.begin(), list.end(), [&](int a, int b2) { return cost[a] > cost[b2]; });
        psst::ClassLaunch c{};
        c.cl = ct[0];
        c.n_nets = (int)list.size();
        long long mx = 0, rows = 0, chunks = 0;
        for (int b : list) {
            mx = std::max(mx, need[b]);
            rows += d->net_neuron_off[b + 1] - d->net_neuron_off[b];
            for (int q = 0; q < ct[0]; ++q) chunks += plans[b].chunks[q];
        }
        c.smem = (int)mx;
        c.block = d->block_threads ? d->block_threads : (ct[1] == 4 ? 256 : ct[1] == 2 ? 512 : 1024);
        c.G = d->row_group ? d->row_group : default_row_group((double)chunks / (double)std::max(1LL, rows));
        if (c.block % c.G) return fail(PSST_ERR_INVALID_ARG, "row_group must divide block_threads");
        ranges.push_back({(int)all_lists.size(), (int)list.size()});
        all_lists.insert(all_lists.end(), list.begin(), list.end());
        h->classes.push_back(c);
    }
    int *dl = nullptr;
    psst::NetPlan *dp = nullptr;
    cudaError_t e = upload(h, &dl, all_lists.data(), all_lists.size());
    if (e == cudaSuccess) e = upload(h, &dp, plans.data(), plans.size());
    for (size_t i = 0; e == cudaSuccess && i < h->classes.size(); ++i) {
        h->classes[i].list = dl + ranges[i].first;
        h->classes[i].plans = dp;
        e = psst::cta_prepare(h->classes[i].cl, max_smem);
    }
    if (e != cudaSuccess) return *err = e, cuda_fail(e, "CTA mode setup");
    // summary for psst_query: the largest class
    h->block = h->classes.empty() ? 0 : h->classes.back().block;
    h->G = h->classes.empty() ? 0 : h->classes.back().G;
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

int psst_create_network(const psst_network_desc *d, psst_net **out) {
    if (!out) return fail(PSST_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int rc = validate(d);
    if (rc) return rc;
    int dev = d->device;
    if (dev < 0 && cudaGetDevice(&dev) != cudaSuccess) return fail(PSST_ERR_CUDA, "no CUDA device");
    DeviceGuard guard(dev);

    const int n_nets = d->n_nets, nt = d->n_syn_types;
    const long long N = d->net_neuron_off[n_nets], S = d->row_ptr[N];
    const int max_smem = psst::cta_max_smem(dev);
    if (max_smem <= 0) return fail(PSST_ERR_CUDA, "cannot query shared memory size of device %d", dev);

    std::vector<int> rowch;
    std::vector<uint8_t> has2;
    row_chunk_counts(d, rowch, has2);
    // cluster sizes needed in CTA mode (0 = does not fit)
    bool all_fit = true;
    for (int b = 0; b < n_nets && all_fit; ++b) {
        const int n0 = d->net_neuron_off[b], Nb = d->net_neuron_off[b + 1] - n0;
        bool fit = false;
        for (int cl = 1; cl <= PSST_MAX_CL && !fit; cl *= 2) {
            if (cl > 1 && Nb < 2 * cl) break;
            std::vector<double> c((size_t)Nb);
            for (int i = 0; i < Nb; ++i) c[i] = rowch[n0 + i];
            std::vector<int> split;
            balanced_split(c, cl, split);
            long long worst = 0;
            for (int q = 0; q < cl; ++q)
                worst = std::max(worst, cta_need(Nb, nt, has2[b], rowch.data() + n0, split[q], split[q + 1]));
            fit = worst <= max_smem;
        }
        all_fit = fit;
    }
    int mode = d->mode;
    if (mode == PSST_MODE_AUTO) mode = all_fit ? PSST_MODE_CTA : PSST_MODE_GRID;
    if (mode == PSST_MODE_GRID && n_nets != 1)
        return fail(PSST_ERR_UNSUPPORTED, "grid mode integrates a single network (got %d)", n_nets);

    psst_net *h = new psst_net();
    h->device = dev;
    h->mode = mode;
    h->block = d->block_threads;
    h->G = d->row_group;
    NetView &v = h->v;
    v.n_nets = n_nets;
    v.n_stypes = nt;
    v.N = N;
    v.S = S;
    v.noise_seed = d->noise_seed;
    v.noise_thresh = d->noise_thresh;
    v.noise_amp = d->noise_amp;
    v.dt = d->dt;
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
        UP(p_fl, has2.data(), n_nets);
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
    rc = mode == PSST_MODE_GRID ? setup_grid(h, d, max_smem, has2[0] != 0, rowch, &e)
                                : setup_cta(h, d, max_smem, rowch, has2, &e);
    if (rc) {
        h->release();
        delete h;
        return rc;
    }
    *out = h;
    return PSST_OK;
}

int psst_integrate(psst_net *h, int64_t n_steps, void *stream) {
    if (!h) return fail(PSST_ERR_INVALID_ARG, "handle is NULL");
    if (n_steps < 0) return fail(PSST_ERR_INVALID_ARG, "n_steps must be >= 0");
    h->launches = 0;
    if (n_steps == 0) return PSST_OK;
    DeviceGuard guard(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    const long long chunk = 1LL << 30;
    for (long long done = 0; done < n_steps;) {
        const int n = (int)std::min<long long>(chunk, n_steps - done);
        if (h->mode == PSST_MODE_GRID) {
            cudaError_t e = psst::grid_launch(h->v, h->gv, h->step + done, n, h->grid, h->block, h->G, h->smem, st);
            if (e != cudaSuccess) return cuda_fail(e, "psst_integrate launch");
            ++h->launches;
        } else {
            for (const psst::ClassLaunch &c : h->classes) {
                cudaError_t e = psst::cta_launch(h->v, c, h->step + done, n, st);
                if (e != cudaSuccess) return cuda_fail(e, "psst_integrate launch");
                ++h->launches;
            }
        }
        done += n;
    }
    h->step += n_steps;
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
    if (!h || !src) return fail(PSST_ERR_INVALID_ARG, "NULL argument");
    const size_t dim = (size_t)(4 * h->v.N + 2 * h->v.S);
    if (n != dim) return fail(PSST_ERR_INVALID_ARG, "src holds %zu floats, state has %zu", n, dim);
    DeviceGuard guard(h->device);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(h->v.state, src, dim * sizeof(float),
                                    src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !src_on_device) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? PSST_OK : cuda_fail(e, "psst_set_state");
}

int psst_set_step(psst_net *h, int64_t step) {
    if (!h) return fail(PSST_ERR_INVALID_ARG, "handle is NULL");
    if (step < 0) return fail(PSST_ERR_INVALID_ARG, "step must be >= 0");
    h->step = step;
    h->rec_reset = step;
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
    out->row_group = h->G;
    out->grid_ctas = h->grid;
    out->smem_bytes = h->smem;
    out->n_single_cta_nets = h->n_smem;
    out->n_cluster_nets = h->n_global;
    out->n_launch_classes = (int32_t)h->classes.size();
    out->kernel_launches = h->launches;
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
