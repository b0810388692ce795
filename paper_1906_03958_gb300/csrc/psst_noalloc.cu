// An entry point for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running under an
// allocator that must not be bypassed (a framework's pool, a memory-capped
// sandbox), or code that only holds buffers handed to it by someone else.
// psst_integrate_grid_noalloc lets them run the grid-wide integration of
// one network on buffers they already own.  The inputs and outputs are the
// caller's device arrays; the only extra memory the kernels need -- the
// double-buffered gate-map tables, the barrier words and the per-CTA plan --
// lives in one fixed-size array in device global memory that is part of this
// library (PSST_NOALLOC_SCRATCH_BYTES), so the call itself allocates nothing.
//
// That array is created when the library is loaded on a device and stays
// there, on every GPU that loads the library, until the process exits.
// Every call uses the same array and finds it as the previous call left it:
// the function clears what must start from zero, and two calls whose GPU
// work overlaps (different streams, no ordering between them) race on it.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "../../include/psst.h"
#include "psst_device.cuh"
#include "psst_internal.h"
#include "psst_syn.cuh"

namespace {

constexpr size_t kScratchBytes = PSST_NOALLOC_SCRATCH_BYTES;
constexpr int kMaxGrid = 512;  // CTAs of one launch (one per SM)

// The scratch array.  Host code sees only a stand-in for its symbol; the
// device address comes from cudaGetSymbolAddress (see scratch_base).
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Scratch layout (byte offsets).
constexpr size_t kOffBar = 0;         // unsigned[2]: the grid barrier's 64-bit arrival count
constexpr size_t kOffFlag = 8;        // unsigned: network holds second-order synapses
constexpr size_t kOffPulse = 16;      // long long[2]: pulse window
constexpr size_t kOffSplit = 256;     // int[kMaxGrid + 1]: first row of each CTA
constexpr size_t kOffItems = kOffSplit + 4 * (kMaxGrid + 1 + 63);  // int[2 * kMaxGrid]
constexpr size_t kOffTables = 8192;   // float2 [2][M], then float4 [2][M]
static_assert(kOffItems + 8 * kMaxGrid <= kOffTables, "scratch header overlaps the tables");

struct DeviceScratch {
    bool ready = false;
    unsigned char *base = nullptr;
};
DeviceScratch g_devices[64];
std::mutex g_setup_mutex;

// Errors of this entry point are reported by return code only (the text
// documents the case); nothing is stored, so nothing is allocated.
inline int err_msg(int code, const char *) { return code; }

// Device address of the scratch array on the current device, looked up once
// per device (the first call on each device does this).
int scratch_base(int dev, unsigned char **out) {
    if (dev < 0 || dev >= 64) return err_msg(PSST_ERR_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceScratch &d = g_devices[dev];
    if (!d.ready) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return err_msg(PSST_ERR_CUDA, cudaGetErrorString(e));
        d.base = (unsigned char *)p;
        d.ready = true;
    }
    *out = d.base;
    return PSST_OK;
}

// Plan of the grid launch, computed on the device from the caller's arrays:
// CTA c owns rows [split[c], split[c+1]) with about equal synapses + 8 per
// row, and counts its first- and second-order work items of K chunks.
__global__ void noalloc_plan_kernel(const long long *row_ptr, const uint32_t *syn_code, const float *sparams,
                                    long long N, int K, long long pulse_on, long long pulse_off,
                                    unsigned char *scratch) {
    int *split = (int *)(scratch + kOffSplit);
    int *items = (int *)(scratch + kOffItems);
    unsigned *flag = (unsigned *)(scratch + kOffFlag);
    __shared__ long long s_lo, s_hi;
    __shared__ int s_i1, s_i2;
    __shared__ unsigned s_has2;
    const int c = blockIdx.x, G = gridDim.x;
    if (threadIdx.x == 0) {
        const double total = (double)row_ptr[N] + 8.0 * (double)N;
        long long bound[2];
        for (int q = 0; q < 2; ++q) {
            const double target = total * (double)(c + q) / (double)G;
            long long lo = 0, hi = N;
            while (lo < hi) {  // first row whose prefix cost reaches the target
                const long long mid = (lo + hi) / 2;
                if ((double)row_ptr[mid] + 8.0 * (double)mid < target) lo = mid + 1;
                else hi = mid;
            }
            bound[q] = lo;
        }
        s_lo = bound[0];
        s_hi = (c == G - 1) ? N : bound[1];
        s_i1 = s_i2 = 0;
        s_has2 = 0;
        split[c] = (int)s_lo;
        if (c == G - 1) split[G] = (int)N;
        if (c == 0) {
            unsigned *bar = (unsigned *)(scratch + kOffBar);
            bar[0] = bar[1] = 0u;
            long long *pw = (long long *)(scratch + kOffPulse);
            pw[0] = pulse_on;
            pw[1] = pulse_off;
        }
    }
    __syncthreads();
    int i1 = 0, i2 = 0;
    unsigned h2 = 0;
    for (long long i = s_lo + threadIdx.x; i < s_hi; i += blockDim.x) {
        int n2 = 0;
        for (long long k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
            n2 += sparams[(syn_code[k] >> 24) * PSST_SYN_NPARAM] != 0.0f;
        const int n1 = (int)(row_ptr[i + 1] - row_ptr[i]) - n2;
        i1 += psst::part_items(n1, K);
        i2 += psst::part_items(n2, K);
        h2 |= n2 != 0;
    }
    atomicAdd(&s_i1, i1);
    atomicAdd(&s_i2, i2);
    atomicOr(&s_has2, h2);
    __syncthreads();
    if (threadIdx.x == 0) {
        items[c] = s_i1;
        items[G + c] = s_i2;
        if (s_has2) atomicOr(flag, 1u);
    }
}

}  // namespace

extern "C" int psst_integrate_grid_noalloc(const psst_device_network *d, int64_t step0, int64_t n_steps,
                                           void *stream) {
    if (!d) return err_msg(PSST_ERR_INVALID_ARG, "network is NULL");
    if (!d->row_ptr || !d->syn_code || !d->weight || !d->neuron_type || !d->neuron_params || !d->syn_params ||
        !d->i_const || !d->state || !d->err)
        return err_msg(PSST_ERR_INVALID_ARG, "a required device pointer is NULL");
    if (d->n_neurons < 1 || d->n_synapses < 0) return err_msg(PSST_ERR_INVALID_ARG, "bad sizes");
    if (d->n_syn_types < 1 || d->n_syn_types > PSST_MAX_SYN_TYPES)
        return err_msg(PSST_ERR_INVALID_ARG, "n_syn_types must be in 1..8");
    if (!(d->dt > 0.0f)) return err_msg(PSST_ERR_INVALID_ARG, "dt must be > 0");
    if (d->rec_stride < 0 || (d->rec_stride > 0 && (!d->rec || d->rec_capacity < 1)))
        return err_msg(PSST_ERR_INVALID_ARG, "recording needs rec and rec_capacity >= 1");
    if (d->noise_thresh > (1u << 24)) return err_msg(PSST_ERR_INVALID_ARG, "noise_thresh must be <= 2^24");
    if (d->item_chunks < 0 || d->item_chunks > 64) return err_msg(PSST_ERR_INVALID_ARG, "item_chunks must be in 0..64");
    if (n_steps < 0 || step0 < 0) return err_msg(PSST_ERR_INVALID_ARG, "step0 and n_steps must be >= 0");
    const long long N = d->n_neurons, M = N * d->n_syn_types;
    if (M >= 65536) return err_msg(PSST_ERR_UNSUPPORTED, "n_neurons x n_syn_types must stay below 65536");
    // gate-map tables: [2][M] float2, and [2][M] float4 for second-order networks
    if (kOffTables + 2 * (size_t)M * 8 > kScratchBytes)
        return err_msg(PSST_ERR_UNSUPPORTED, "network too large for the fixed scratch array");
    if (n_steps == 0) return PSST_OK;

    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return err_msg(PSST_ERR_CUDA, cudaGetErrorString(e));
    unsigned char *scratch = nullptr;
    int rc = scratch_base(dev, &scratch);
    if (rc) return rc;
    int sms = 0, optin = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return err_msg(PSST_ERR_CUDA, "device attributes");
    const int max_dyn = optin - psst::cta_static_smem() - 64;
    const int G = (int)std::max(1LL, std::min<long long>(std::min(sms, kMaxGrid), (N + 7) / 8));
    int K = d->item_chunks;
    if (K == 0) {
        const long long chunks = (d->n_synapses / 4 + N) / G + 1;
        K = (int)std::max(1LL, std::min(8LL, (chunks + 767) / 768));
    }
    cudaStream_t st = (cudaStream_t)stream;

    // plan on the device, then check every CTA's shared memory on the host
    e = cudaMemsetAsync(scratch + kOffFlag, 0, sizeof(unsigned), st);
    if (e == cudaSuccess) {
        noalloc_plan_kernel<<<G, 256, 0, st>>>((const long long *)d->row_ptr, d->syn_code, d->syn_params, N, K, d->pulse_on,
                                               d->pulse_off, scratch);
        e = cudaGetLastError();
    }
    int split[kMaxGrid + 1], items[2 * kMaxGrid];
    unsigned has2 = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(split, scratch + kOffSplit, sizeof(int) * (G + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(items, scratch + kOffItems, sizeof(int) * 2 * G, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&has2, scratch + kOffFlag, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return err_msg(PSST_ERR_CUDA, cudaGetErrorString(e));
    if (has2 && kOffTables + 2 * (size_t)M * (8 + 16) > kScratchBytes)
        return err_msg(PSST_ERR_UNSUPPORTED, "second-order network too large for the fixed scratch array");
    for (int c = 0; c < G; ++c) {
        const int n = split[c + 1] - split[c];
        const long long need = psst::make_nlayout(n, n, n * d->n_syn_types, has2 != 0).syn +
                               psst::items_smem_bytes(items[c], items[G + c], K, n, has2 != 0);
        if (need > max_dyn) return err_msg(PSST_ERR_UNSUPPORTED, "a CTA's share exceeds shared memory");
    }

    psst::NetView v{};
    v.n_nets = 1;
    v.n_stypes = d->n_syn_types;
    v.N = N;
    v.S = d->n_synapses;
    v.row_ptr = (const long long *)d->row_ptr;
    v.syn_code = d->syn_code;
    v.weight = d->weight;
    v.neuron_type = d->neuron_type;
    v.nparams = d->neuron_params;
    v.sparams = d->syn_params;
    v.i_const = d->i_const;
    v.pulse_amp = d->pulse_amp;
    v.pulse_on = (const long long *)(scratch + kOffPulse);
    v.pulse_off = (const long long *)(scratch + kOffPulse) + 1;
    v.noise_seed = d->noise_seed;
    v.noise_thresh = d->noise_thresh;
    v.noise_amp = d->noise_amp;
    v.dt = d->dt;
    v.state = d->state;
    v.rec = d->rec;
    v.rec_stride = d->rec_stride;
    v.rec_cap = d->rec_stride > 0 ? d->rec_capacity : 0;
    v.net_flags = (const uint8_t *)(scratch + kOffFlag);  // low byte of the flag word
    v.err = d->err;
    psst::GridView g{};
    g.c1 = (float2 *)(scratch + kOffTables);
    g.c2 = has2 ? (float4 *)(scratch + kOffTables + 2 * (size_t)M * 8) : nullptr;
    g.bar = (unsigned *)(scratch + kOffBar);
    g.row_split = (const int *)(scratch + kOffSplit);
    g.items = (const int *)(scratch + kOffItems);
    g.K = K;
    g.timeout_ns = 2000000000ULL;

    int per_sm = 0;
    e = psst::grid_occupancy(1024, max_dyn, &per_sm);
    if (e != cudaSuccess) return err_msg(PSST_ERR_CUDA, cudaGetErrorString(e));
    if (per_sm < 1) return err_msg(PSST_ERR_UNSUPPORTED, "grid kernel does not fit an SM");
    for (long long done = 0; done < n_steps;) {
        const int n = (int)std::min<long long>(1LL << 30, n_steps - done);
        e = psst::grid_launch(v, g, step0 + done, n, G, 1024, max_dyn, st);
        if (e != cudaSuccess) return err_msg(PSST_ERR_CUDA, cudaGetErrorString(e));
        done += n;
    }
    return PSST_OK;
}
