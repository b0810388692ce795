// C interface (include/psst.h): validation, device layout, launches.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/psst.h"
#include "psst_internal.h"

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

// Lanes per CSR row: the power of two nearest half the mean row length,
// clamped to 4..32.
int default_row_group(double mean_row) {
    int g = 4;
    while (g < 32 && g < mean_row * 0.5) g <<= 1;
    return g;
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
    psst_net *h = new psst_net();
    h->device = dev;
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

    // per-synapse code and per-network flags, work order
    std::vector<uint32_t> code((size_t)S);
    std::vector<uint8_t> flags((size_t)n_nets, 0);
    std::vector<int> order((size_t)n_nets);
    std::vector<double> cost((size_t)n_nets);
    int max_smem = psst::cta_max_smem(dev);
    if (max_smem <= 0) {
        delete h;
        return fail(PSST_ERR_CUDA, "cannot query shared memory size");
    }
    int need_smem = 0;
    int n_smem = 0, n_global = 0;
    long long max_n = 0;
    bool any_over = false;
    for (int b = 0; b < n_nets; ++b) {
        const long long n0 = d->net_neuron_off[b], n1 = d->net_neuron_off[b + 1];
        const long long s0 = d->row_ptr[n0], s1 = d->row_ptr[n1];
        bool has2 = false;
        for (long long k = s0; k < s1; ++k) {
            const int t = d->syn_type[k];
            code[k] = ((uint32_t)t << 24) | (uint32_t)(d->pre[k] * nt + t);
            has2 |= d->syn_params[(size_t)t * PSST_SYN_NPARAM] == 1.0f;
        }
        const int nb = (int)(n1 - n0), sb = (int)(s1 - s0);
        max_n = std::max<long long>(max_n, nb);
        const psst::Layout full = psst::make_layout(nb, sb, nt, has2, true);
        const psst::Layout part = psst::make_layout(nb, sb, nt, has2, false);
        uint8_t f = has2 ? psst::NET_HAS2 : 0;
        if (full.total <= max_smem) {
            f |= psst::NET_FITS_SMEM;
            need_smem = std::max(need_smem, full.total);
            ++n_smem;
        } else {
            need_smem = std::max(need_smem, part.total);
            any_over |= part.total > max_smem;
            ++n_global;
        }
        flags[b] = f;
        order[b] = b;
        cost[b] = (double)sb + 40.0 * nb;
    }
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost[a] > cost[b]; });

    int mode = d->mode;
    if (mode == PSST_MODE_AUTO) mode = PSST_MODE_CTA;
    if (mode == PSST_MODE_GRID) {
        delete h;
        return fail(PSST_ERR_UNSUPPORTED, "grid mode is not available in this build");
    }
    if (any_over) {
        delete h;
        return fail(PSST_ERR_UNSUPPORTED, "a network has too many neurons for one CTA (max %lld)", max_n);
    }
    h->mode = mode;
    h->n_smem = n_smem;
    h->n_global = n_global;
    h->smem = need_smem;
    h->block = d->block_threads ? d->block_threads : 512;
    const double mean_row = N ? (double)S / (double)N : 0.0;
    h->G = d->row_group ? d->row_group : default_row_group(mean_row);
    if (h->G > 32 || h->block % h->G) {
        delete h;
        return fail(PSST_ERR_INVALID_ARG, "row_group must divide block_threads");
    }

    // device arrays
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
        int *p_off, *p_nt, *p_order;
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
        UP(p_order, order.data(), n_nets);
        UP(p_fl, flags.data(), n_nets);
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
        v.order = p_order;
        v.net_flags = p_fl;
    }
#undef UP
    const long long dim = 4 * N + 2 * S;
    if (e == cudaSuccess) e = h->alloc(&v.state, (size_t)dim);
    if (e == cudaSuccess && v.rec_cap > 0) e = h->alloc(&v.rec, (size_t)(v.rec_cap * N));
    if (e == cudaSuccess) e = h->alloc(&v.work_counter, 4);
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
    if (e == cudaSuccess) {
        int per_sm = 0, sms = 0;
        e = psst::cta_occupancy(h->block, h->smem, &per_sm);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e == cudaSuccess && per_sm < 1) {
            h->release();
            delete h;
            return fail(PSST_ERR_UNSUPPORTED, "block of %d threads with %d B shared memory cannot launch",
                        d->block_threads ? d->block_threads : 512, need_smem);
        }
        h->grid = (int)std::min<long long>(n_nets, (long long)per_sm * sms);
    }
    if (e != cudaSuccess) {
        h->release();
        delete h;
        return cuda_fail(e, "psst_create_network");
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
        cudaError_t e = psst::cta_launch(h->v, h->step + done, n, h->grid, h->block, h->G, h->smem, st);
        if (e != cudaSuccess) return cuda_fail(e, "psst_integrate launch");
        ++h->launches;
        done += n;
    }
    h->step += n_steps;
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
    out->n_smem_nets = h->n_smem;
    out->n_global_nets = h->n_global;
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
