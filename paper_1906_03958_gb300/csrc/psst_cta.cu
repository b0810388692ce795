// Network-resident RK4 integration for batches of small and medium networks.
//
// One network is owned by a cluster of CL CTAs (CL = 1, 2 or 4, chosen per
// network by its shared-memory footprint) for all of a launch's steps.  Each
// CTA of the cluster holds every neuron of the network and the synapses of
// its own block of CSR rows (postsynaptic neurons) in shared memory.  One
// launch per size class integrates all networks of that class; blocks are
// ordered largest network first.
//
// Per RK4 step (classic tableau, Sec. "Brain simulations as computational
// graphs", RK4 paragraph) and stage s = 0..3:
//   S-phase: synaptic current of the CTA's own rows at stage s (padded
//            4-wide chunks, see psst_syn.cuh); each row's value is written to
//            every CTA of the cluster (distributed shared memory);
//   barrier: CTA barrier (CL = 1) or cluster barrier (CL > 1);
//   N-phase: every CTA evaluates the HH right-hand side of all N neurons and
//            the gate maps of all (presynaptic neuron, type) pairs -- the same
//            values in every CTA, so nothing else has to be exchanged;
//   barrier: CTA barrier.
// The synaptic current is double-buffered by stage parity so a fast CTA can
// write the next stage's values while a peer still reads this stage's.
//
// Synaptic gates: a gate's equation dr/dt = a T_j (1 - r) - b r is affine in
// r with coefficients set by its presynaptic neuron j alone, so each RK4
// stage value is r^(s) = P_s[j] + Q_s[j] r0 (second-order pairs:
// s^(s) = U_s + X_s r0 + Z_s s0) with the maps propagated once per
// (neuron, type) and stage; the step-end map is applied lazily at the next
// step's first stage.  This evaluates the same RK4 map as the textbook stage
// recursion, with each synapse costing one FMA per stage.
#include <cuda_runtime.h>

#include "psst_device.cuh"
#include "psst_internal.h"
#include "psst_syn.cuh"

namespace psst {

namespace {

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void st_peer(float *local, unsigned rank, float x) {
    const unsigned laddr = (unsigned)__cvta_generic_to_shared(local);
    unsigned raddr;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(raddr) : "r"(laddr), "r"(rank));
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(raddr), "f"(x) : "memory");
}

struct SmemCoef {
    const float2 *t1;
    const float4 *t2;
    __device__ __forceinline__ float2 r(int i) const { return t1[i]; }
    __device__ __forceinline__ float4 s(int i) const { return t2[i]; }
};

template <int CL>
struct IsynOut {
    float *isyn;  // this stage's buffer, indexed by network row
    int r_lo;
    unsigned rank;
    __device__ __forceinline__ void operator()(int row, float x) const {
        float *p = isyn + r_lo + row;
        *p = x;
        if (CL > 1) {
#pragma unroll
            for (unsigned q = 1; q < CL; ++q) st_peer(p, (rank + q) % CL, x);
        }
    }
};

template <int CL, bool HAS2>
__device__ void run_net(const NetView &v, int b, const NetPlan &pl, long long step0, int nsteps, int G,
                        unsigned char *smem, const float *stab) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const unsigned rank = CL > 1 ? cluster_rank() : 0u;
    const int n0 = v.net_off[b], N = v.net_off[b + 1] - n0;
    const int nt = v.n_stypes, M = N * nt;
    const long long sbase = v.row_ptr[n0];
    const int r_lo = pl.split[rank], nrows = pl.split[rank + 1] - r_lo;
    const NeuronLayout L = make_nlayout(N, nt, HAS2, nrows);
    float *y0 = (float *)(smem + L.y0), *ys = (float *)(smem + L.ys), *acc = (float *)(smem + L.acc);
    float *prm = (float *)(smem + L.prm), *iext = (float *)(smem + L.iext);
    float *isyn = (float *)(smem + L.isyn), *vst = (float *)(smem + L.vst);
    float2 *cur1 = (float2 *)(smem + L.cur1), *acc1 = (float2 *)(smem + L.acc1), *fin1 = (float2 *)(smem + L.fin1);
    float4 *cur2 = HAS2 ? (float4 *)(smem + L.cur2) : nullptr;
    float4 *acc2 = HAS2 ? (float4 *)(smem + L.acc2) : nullptr;
    float4 *fin2 = HAS2 ? (float4 *)(smem + L.fin2) : nullptr;
    int *tmp = (int *)(smem + L.tmp);
    RowChunks rc = carve_rows(smem + L.syn, nrows, pl.chunks[rank], HAS2);

    float *gV = v.state + n0;
    float *gr = v.state + 4 * v.N + sbase;
    float *gs = v.state + 4 * v.N + v.S + sbase;
    const float *gw = v.weight + sbase;
    const uint32_t *gcode = v.syn_code + sbase;

    for (int i = tid; i < N; i += nthr) {
        const float V = gV[i];
        y0[i] = V;
        vst[i] = V;  // stage-0 potential, parity 0
#pragma unroll
        for (int x = 1; x < 4; ++x) {
            const float y = gV[(long long)x * v.N + i];
            y0[x * N + i] = y;
            ys[x * N + i] = y;
        }
        const float *p = v.nparams + (long long)v.neuron_type[n0 + i] * PSST_NEURON_NPARAM;
        prm[NP_C * N + i] = 1.0f / p[NP_C];
#pragma unroll
        for (int x = 1; x < PSST_NEURON_NPARAM; ++x) prm[x * N + i] = p[x];
    }
    for (int k = tid; k < M; k += nthr) {
        fin1[k] = make_float2(0.0f, 1.0f);
        if (HAS2) {
            const float *sp = stab + (k % nt) * 9;
            fin2[k] = make_float4(0.0f, 0.0f, 1.0f, sp[SP_KIND] != 0.0f ? sp[SP_KD] : 1.0f);
        }
    }
    load_rows<HAS2>(rc, v, n0, sbase, r_lo, gr, gs, gw, gcode, stab, tmp);  // ends with __syncthreads
    if (CL > 1) cluster_sync();

    const float dt = v.dt;
    // coefficient pairs are taken by the threads after the neuron threads
    int tq = tid - N % nthr;
    if (tq < 0) tq += nthr;

    for (int it = 0; it < nsteps; ++it) {
        const long long step = step0 + it;
        for (int i = tid; i < N; i += nthr) iext[i] = input_current(v, b, (long long)n0 + i, step);
#define PSST_STAGE(ST)                                                                                     \
    {                                                                                                      \
        const float *vcur = vst + (ST & 1) * N;                                                            \
        float *vnxt = vst + ((ST + 1) & 1) * N;                                                            \
        float *isy = isyn + (ST & 1) * N;                                                                  \
        const SmemCoef cf{ST == 0 ? fin1 : cur1, ST == 0 ? fin2 : cur2};                                   \
        sphase<ST, HAS2>(rc, vcur + r_lo, cf, G, IsynOut<CL>{isy, r_lo, rank});                            \
        if (CL > 1) cluster_sync();                                                                        \
        else __syncthreads();                                                                              \
        for (int i = tid; i < N; i += nthr) {                                                              \
            const float vn = neuron_update<ST>(i, N, vcur[i], y0, acc, ys, prm, iext[i], isy[i], dt);      \
            vnxt[i] = vn;                                                                                  \
            if (ST == 3 && rank == 0 && v.rec_stride > 0 && ((step + 1) % v.rec_stride) == 0) {            \
                const long long frame = (step + 1) / v.rec_stride - 1;                                     \
                v.rec[(frame % v.rec_cap) * v.N + n0 + i] = vn;                                            \
            }                                                                                              \
        }                                                                                                  \
        for (int p = tq; p < M; p += nthr) {                                                               \
            float4 d4 = make_float4(0.f, 0.f, 0.f, 0.f);                                                   \
            float4 &c2 = HAS2 ? cur2[p] : d4;                                                              \
            float4 &a2 = HAS2 ? acc2[p] : d4;                                                              \
            float4 &f2 = HAS2 ? fin2[p] : d4;                                                              \
            coef_update<ST, HAS2>(stab + (p % nt) * 9, vcur[p / nt], dt, cur1[p], acc1[p], fin1[p], c2, a2, \
                                  f2);                                                                     \
        }                                                                                                  \
        __syncthreads();                                                                                   \
    }
        PSST_STAGE(0)
        PSST_STAGE(1)
        PSST_STAGE(2)
        PSST_STAGE(3)
#undef PSST_STAGE
    }

    // write back: own synapses with the last step's gate map; neurons by rank 0
    struct Fin {
        const float2 *f1;
        const float4 *f2;
        __device__ __forceinline__ float2 r(int i) const { return f1[i]; }
        __device__ __forceinline__ float4 s(int i) const { return f2[i]; }
    } fin{fin1, fin2};
    store_rows<HAS2>(rc, v, n0, sbase, r_lo, gr, gs, gcode, stab, fin);
    if (rank == 0) {
        bool bad = false;
        for (int i = tid; i < N; i += nthr) {
#pragma unroll
            for (int x = 0; x < 4; ++x) {
                const float y = y0[x * N + i];
                bad |= !isfinite(y);
                gV[(long long)x * v.N + i] = y;
            }
        }
        if (bad) set_error(v.err, PSST_ERR_NONFINITE);
    }
    if (CL > 1) cluster_sync();  // no CTA leaves while a peer may still write into it
}

template <int CL>
__global__ void __launch_bounds__(1024) net_kernel(NetView v, const int *list, const NetPlan *plans,
                                                   long long step0, int nsteps, int G) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float stab[PSST_MAX_SYN_TYPES * PSST_SYN_NPARAM];
    for (int i = threadIdx.x; i < v.n_stypes * PSST_SYN_NPARAM; i += blockDim.x) {
        float x = v.sparams[i];
        if (i % PSST_SYN_NPARAM == SP_KP) x = 1.0f / x;  // stored as 1/Kp
        stab[i] = x;
    }
    __syncthreads();
    const int b = list[blockIdx.x / CL];
    if (v.net_flags[b] & NET_HAS2) run_net<CL, true>(v, b, plans[b], step0, nsteps, G, smem, stab);
    else run_net<CL, false>(v, b, plans[b], step0, nsteps, G, smem, stab);
}

template <int CL>
cudaError_t launch_cl(const NetView &v, const ClassLaunch &c, long long step0, int nsteps, cudaStream_t stream) {
    if (CL == 1) {
        net_kernel<1><<<c.n_nets, c.block, c.smem, stream>>>(v, c.list, c.plans, step0, nsteps, c.G);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c.n_nets * CL);
    cfg.blockDim = dim3(c.block);
    cfg.dynamicSmemBytes = (size_t)c.smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = CL;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, net_kernel<CL>, v, c.list, c.plans, step0, nsteps, c.G);
}

}  // namespace

int cta_max_smem(int device) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess) return -1;
    return v - (int)(PSST_MAX_SYN_TYPES * PSST_SYN_NPARAM * sizeof(float) + 64);
}

cudaError_t cta_prepare(int cl, int max_smem) {
    const void *k = cl == 1 ? (const void *)net_kernel<1> : cl == 2 ? (const void *)net_kernel<2>
                                                                    : (const void *)net_kernel<4>;
    // the attribute is an upper bound shared by every launch of this kernel
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem);
    if (e == cudaSuccess && cl > 1) e = cudaFuncSetAttribute(k, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

cudaError_t cta_launch(const NetView &v, const ClassLaunch &c, long long step0, int nsteps, cudaStream_t stream) {
    switch (c.cl) {
    case 1: return launch_cl<1>(v, c, step0, nsteps, stream);
    case 2: return launch_cl<2>(v, c, step0, nsteps, stream);
    case 4: return launch_cl<4>(v, c, step0, nsteps, stream);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace psst
