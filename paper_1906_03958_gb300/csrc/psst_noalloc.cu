// An entry point for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code running under an
// allocator that must not be bypassed (a framework's pool, a memory-capped
// sandbox), or code that only holds buffers handed to it by someone else.
// psst_integrate_grid_noalloc lets them run the grid-wide integration of
// one network on buffers they already own.  The inputs and outputs are the
// caller's device arrays; the only extra memory the kernels need -- the
// double-buffered gate-map tables, the per-CTA phase flags and the plan --
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
constexpr size_t kOffFlag = 8;        // unsigned: network holds second-order synapses
constexpr size_t kOffBad = 12;        // unsigned: bits of the array checks that failed (1 row_ptr, 2 syn_code, 4 neuron_type)
constexpr size_t kOffPulse = 16;      // long long[2]: pulse window
constexpr size_t kOffK = 32;          // int: chunks per work item of the launch
constexpr size_t kOffSplit = 256;     // int[kMaxGrid + 1]: first row of each CTA
constexpr size_t kOffItems = kOffSplit + 4 * (kMaxGrid + 1 + 63);  // int[2 * kMaxGrid]
constexpr size_t kOffPhase = 8192;    // unsigned long long[kMaxGrid][GRID_FLAG_STRIDE]: each CTA's published phase
constexpr size_t kOffTables = kOffPhase + 8 * kMaxGrid * psst::GRID_FLAG_STRIDE;  // float2 [2][M], then float4 [2][M]
// Planning only (dead before the integration launch, which reuses the
// space for its tables): per row n1, n2 (int[N] each), then the prefix of
// the row costs (long long[N + 1]).
constexpr size_t kOffRows = kOffTables;
static_assert(kOffItems + 8 * kMaxGrid <= kOffPhase, "scratch header overlaps the phase flags");
static_assert(kOffRows + 16 * 65536 + 8 <= kScratchBytes, "planning arrays exceed the scratch array");

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

// Array checks and per-row counts, one thread per row: row_ptr must rise
// from 0 to n_synapses; each syn_code must carry a type below n_syn_types,
// a pair index pre * n_syn_types + type with that same type and pre < N;
// each neuron_type must index the neuron table.  A failed check sets its
// bit in the scratch word kOffBad (and the rest of the call is skipped);
// nothing outside the arrays' stated extents is read, whatever they hold.
// Row i's first- and second-order synapse counts go to n1[i], n2[i].
__global__ void noalloc_rows_kernel(const long long *row_ptr, const uint32_t *syn_code, const int *neuron_type,
                                    const float *sparams, long long N, long long S, int nt, int n_ntypes,
                                    unsigned char *scratch) {
    int *n1a = (int *)(scratch + kOffRows), *n2a = n1a + N;
    unsigned bad = 0, h2 = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        long long a = row_ptr[i], b = row_ptr[i + 1];
        if ((i == 0 && a != 0) || (i == N - 1 && b != S)) bad |= 1u;
        if (a < 0 || b < a || b > S) {
            bad |= 1u;
            a = b = 0;
        }
        int n2 = 0;
        for (long long k = a; k < b; ++k) {
            const uint32_t code = syn_code[k];
            const unsigned t = code >> 24, idx = code & 0xFFFFFFu;
            if (t >= (unsigned)nt || idx % (unsigned)nt != t || (long long)(idx / (unsigned)nt) >= N) {
                bad |= 2u;
                continue;
            }
            n2 += sparams[t * PSST_SYN_NPARAM + psst::SP_KIND] != 0.0f;
        }
        const int ty = neuron_type[i];
        if (ty < 0 || ty >= n_ntypes) bad |= 4u;
        n1a[i] = (int)(b - a) - n2;
        n2a[i] = n2;
        h2 |= n2 != 0;
    }
    if (bad) atomicOr((unsigned *)(scratch + kOffBad), bad);
    if (h2) atomicOr((unsigned *)(scratch + kOffFlag), 1u);
}

// Plan of the grid launch (one CTA of PLAN_THREADS threads), the same as
// psst_integrate's grid mode with one gate per synapse: row i costs its
// 4-synapse chunks of each order plus 2; CTA c owns the rows up to the
// first whose cost prefix reaches c/G of the total; without a caller's K,
// K = ceil(largest CTA's chunks / 768), clamped to 1..8; then each CTA's
// first- and second-order work items of K chunks.
constexpr int PLAN_THREADS = 1024;

__global__ void __launch_bounds__(PLAN_THREADS) noalloc_plan_kernel(long long N, int G, int user_K, long long pulse_on,
                                                                   long long pulse_off, unsigned char *scratch) {
    if (*(volatile unsigned *)(scratch + kOffBad) != 0) return;  // arrays rejected: plan nothing
    const int *n1a = (const int *)(scratch + kOffRows), *n2a = n1a + N;
    long long *pref = (long long *)(scratch + kOffRows + 8 * N);
    int *split = (int *)(scratch + kOffSplit);
    int *items = (int *)(scratch + kOffItems);
    __shared__ long long s_part[PLAN_THREADS];
    __shared__ long long s_worst;
    const int tid = threadIdx.x;
    auto row_chunks = [&](long long i) -> long long { return (n1a[i] + 3) / 4 + (n2a[i] + 3) / 4; };
    // cost prefix: thread t sums a contiguous block of rows, then a block scan
    const long long R = (N + PLAN_THREADS - 1) / PLAN_THREADS;
    const long long r0 = tid * R < N ? tid * R : N, r1 = r0 + R < N ? r0 + R : N;
    long long sum = 0;
    for (long long i = r0; i < r1; ++i) sum += row_chunks(i) + 2;
    s_part[tid] = sum;
    __syncthreads();
    for (int off = 1; off < PLAN_THREADS; off <<= 1) {  // inclusive Hillis-Steele scan
        const long long x = tid >= off ? s_part[tid - off] : 0;
        __syncthreads();
        s_part[tid] += x;
        __syncthreads();
    }
    long long run = s_part[tid] - sum;
    for (long long i = r0; i < r1; ++i) {
        pref[i] = run;
        run += row_chunks(i) + 2;
    }
    if (tid == PLAN_THREADS - 1) pref[N] = s_part[tid];
    if (tid == 0) s_worst = 0;
    __syncthreads();
    const double total = (double)pref[N];
    for (int c = tid; c <= G; c += PLAN_THREADS) {
        long long lo = 0;
        if (c == G) {
            lo = N;
        } else if (c > 0) {
            const double target = total * c / G;
            long long hi = N;
            while (lo < hi) {  // first row whose cost prefix reaches the target
                const long long mid = (lo + hi) / 2;
                if ((double)pref[mid] < target) lo = mid + 1;
                else hi = mid;
            }
        }
        split[c] = (int)lo;
    }
    __syncthreads();
    for (int c = tid; c < G; c += PLAN_THREADS) {
        const long long a = split[c], b = split[c + 1];
        atomicMax((unsigned long long *)&s_worst, (unsigned long long)(pref[b] - pref[a] - 2 * (b - a)));
    }
    __syncthreads();
    const long long kw = (s_worst + 767) / 768;
    const int K = user_K > 0 ? user_K : (int)(kw < 1 ? 1 : kw > 8 ? 8 : kw);
    // work items per CTA: warp w takes CTAs w, w + 32, ...
    const int lane = tid & 31, warp = tid >> 5;
    for (int c = warp; c < G; c += PLAN_THREADS / 32) {
        int i1 = 0, i2 = 0;
        for (int i = split[c] + lane; i < split[c + 1]; i += 32) {
            i1 += psst::part_items(n1a[i], K);
            i2 += psst::part_items(n2a[i], K);
        }
        for (int o = 16; o > 0; o >>= 1) {
            i1 += __shfl_xor_sync(0xffffffffu, i1, o);
            i2 += __shfl_xor_sync(0xffffffffu, i2, o);
        }
        if (lane == 0) {
            items[c] = i1;
            items[G + c] = i2;
        }
    }
    if (tid == 0) {
        *(int *)(scratch + kOffK) = K;
        long long *pw = (long long *)(scratch + kOffPulse);
        pw[0] = pulse_on;
        pw[1] = pulse_off;
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
    if (d->n_neuron_types < 1) return err_msg(PSST_ERR_INVALID_ARG, "n_neuron_types must be >= 1");
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
    cudaStream_t st = (cudaStream_t)stream;

    // check the arrays and plan on the device, then check every CTA's shared
    // memory on the host
    e = cudaMemsetAsync(scratch + kOffFlag, 0, 2 * sizeof(unsigned), st);  // flag and check words
    if (e == cudaSuccess) {
        const int rows_grid = (int)std::max(1LL, std::min<long long>(4LL * sms, (N + 255) / 256));
        noalloc_rows_kernel<<<rows_grid, 256, 0, st>>>((const long long *)d->row_ptr, d->syn_code, d->neuron_type,
                                                       d->syn_params, N, d->n_synapses, d->n_syn_types,
                                                       d->n_neuron_types, scratch);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        noalloc_plan_kernel<<<1, PLAN_THREADS, 0, st>>>(N, G, d->item_chunks, d->pulse_on, d->pulse_off, scratch);
        e = cudaGetLastError();
    }
    int split[kMaxGrid + 1], items[2 * kMaxGrid];
    unsigned words[2] = {0u, 0u};  // has2, failed checks
    int K = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(words, scratch + kOffFlag, sizeof(words), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&K, scratch + kOffK, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(split, scratch + kOffSplit, sizeof(int) * (G + 1), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(items, scratch + kOffItems, sizeof(int) * 2 * G, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return err_msg(PSST_ERR_CUDA, cudaGetErrorString(e));
    if (words[1] != 0u) return err_msg(PSST_ERR_INVALID_ARG, "row_ptr, syn_code or neuron_type out of range");
    const unsigned has2 = words[0];
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
    g.flag = (unsigned long long *)(scratch + kOffPhase);
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
