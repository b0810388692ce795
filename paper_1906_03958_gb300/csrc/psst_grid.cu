// Grid-wide RK4 integration of one large network (cooperative launch, one
// CTA per SM).  CTA c owns a contiguous block of CSR rows (postsynaptic
// neurons) chosen by the host to balance synapse chunks; its neurons and its
// rows' synapses stay in shared memory for the whole launch (4-wide chunk
// layout of psst_syn.cuh).
//
// The only data every CTA needs from the others is, per presynaptic neuron
// and synapse type, the affine gate map of the next stage (psst_cta.cu
// explains the gate formulation).  Each CTA writes the maps of its own
// neurons to a double-buffered table in global memory and reads the whole
// table through L2; one device-wide barrier per RK4 stage separates writers
// from readers, and double buffering removes the write-after-read hazard.
// The barrier spins with a time limit: on expiry it records
// PSST_ERR_TIMEOUT and every CTA returns.
//
// Per-pair variant (all gates of each (presynaptic neuron, type) pair equal,
// as from rest): the owner of a presynaptic neuron keeps its pairs' gate
// state and writes each used pair's next-stage gate value (4 bytes) to a
// compact global table; every CTA copies that table into shared memory with
// coalesced loads once per stage and gathers its synapses' gates from there,
// instead of gathering an 8-byte map per synapse from L2.  Results are
// bitwise equal to the per-synapse variant.
#include <cuda_runtime.h>

#include "psst_device.cuh"
#include "psst_internal.h"
#include "psst_syn.cuh"

namespace psst {

namespace {

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned long long ld_acquire64(const unsigned long long *p) {
    unsigned long long x;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(x) : "l"(p) : "memory");
    return x;
}

// Device-wide barrier over gridDim.x co-resident CTAs, in two halves so
// that work on a CTA's own data can run while the others arrive.  bar holds
// a 64-bit arrival count, zeroed before each launch, that only grows:
// barrier k of a launch is passed when the count reaches (k + 1) gridDim.x,
// and the count a CTA finds on arriving tells it k.  Every grid_arrive is
// followed by its grid_wait before the CTA arrives again, so no CTA arrives
// at barrier k + 1 before all have arrived at k.
//
// grid_arrive: after the phase's global writes; returns the count to wait
// for (in thread 0).
__device__ unsigned long long grid_arrive(unsigned *bar) {
    __syncthreads();
    unsigned long long target = 0;
    if (threadIdx.x == 0) {
        const unsigned long long G = gridDim.x;
        __threadfence();
        const unsigned long long prev = atomicAdd(reinterpret_cast<unsigned long long *>(bar), 1ull);
        target = (prev / G + 1) * G;
    }
    return target;
}

// grid_wait: before the next phase's global reads.  Returns false (after
// recording the error) when the wait ran out of time or another CTA already
// failed.
__device__ bool grid_wait(unsigned *bar, unsigned long long target, unsigned long long timeout_ns, int *err) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        const unsigned long long *cnt = reinterpret_cast<const unsigned long long *>(bar);
        int ok = 1;
        const unsigned long long t0 = globaltimer();
        while (ld_acquire64(cnt) < target) {
            if (*(volatile int *)err != 0) {
                ok = 0;
                break;
            }
            if (globaltimer() - t0 > timeout_ns) {
                set_error(err, PSST_ERR_TIMEOUT);
                ok = 0;
                break;
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

__device__ bool grid_barrier(unsigned *bar, unsigned long long timeout_ns, int *err) {
    return grid_wait(bar, grid_arrive(bar), timeout_ns, err);
}

struct GlobalCoef {
    const float2 *t1;
    const float4 *t2;
    __device__ __forceinline__ float2 r(int i) const { return __ldcg(t1 + i); }
    __device__ __forceinline__ float4 s(int i) const { return __ldcg(t2 + i); }
};

// One stage sg of the handle's method (flags and coefficients at run time:
// one copy of this code serves every stage of RK4, Euler and a tableau);
// par selects the double-buffered potentials, gates and global tables this
// stage reads (the parity of the stage's index counted over the launch).  On
// entry the owned neurons' gates m, h, n of this stage are done and tgt is
// the barrier count to wait for; on return the CTA has arrived at the
// stage's closing barrier (tgt updated) and, when `more`, computed the next
// stage's (sx's) gates.
template <bool HAS2, bool PAIR>
__device__ __forceinline__ bool grid_stage(const NetView &v, const GridView &g, const StageRT &sg,
                                           const StageRT &sx, const Items &it, int lo, int N, int nt, int M,
                                           long long rec_slot, float *vst, float *y0, float *ylo, float *acc,
                                           float *ys,
                                           const float *prm, const float *iext, float2 *cur1, float2 *acc1,
                                           float4 *cur2, float4 *acc2, float *pst, float *gtab, const float *stab,
                                           int par, unsigned long long &tgt, bool more) {
    const bool LAST = sg.last;
    const int tid = threadIdx.x, nthr = blockDim.x, Mloc = N * nt;
    const float *vcur = vst + par * N;
    float *vnxt = vst + (par ^ 1) * N;
    const float *ysc = ys + par * 3 * N;
    float *ysn = ys + (par ^ 1) * 3 * N;
    // the other CTAs' gates and maps of this stage are published
    if (!grid_wait(g.bar, tgt, g.timeout_ns, v.err)) return false;
    if (PAIR) {
        // this stage's gate of every used pair, written by the owners before the last barrier
        const float4 *src = (const float4 *)(g.gt + (size_t)par * g.mt);
        float4 *dst = (float4 *)gtab;
        const int n4 = g.mt >> 2;
#pragma unroll 4
        for (int q = tid; q < n4; q += nthr) dst[q] = __ldcg(src + q);
        __syncthreads();
        sphase_pair(it, gtab, 0);
    } else {
        sphase<HAS2>(sg.first, it, GlobalCoef{g.c1 + (size_t)par * M, HAS2 ? g.c2 + (size_t)par * M : nullptr});
    }
    __syncthreads();
    // independent work units: potential of each owned neuron and the gate map
    // of each own (neuron, type) pair; the potentials take whole warps
    float *r0p = pst, *s0p = pst + Mloc, *r0lo = pst + 2 * Mloc, *s0lo = pst + 3 * Mloc;
    float *gout = PAIR ? g.gt + (size_t)(par ^ 1) * g.mt : nullptr;
    float2 *o1 = g.c1 + (size_t)(par ^ 1) * M + (size_t)lo * nt;
    float4 *o2 = HAS2 ? g.c2 + (size_t)(par ^ 1) * M + (size_t)lo * nt : nullptr;
    const int nw = (N + 31) & ~31;
    const int U = nw + Mloc;
    for (int u = tid; u < U; u += nthr) {
        if (u < nw) {
            // the whole warp takes this branch (nw and nthr are multiples of 32)
            const bool own = u < N;
            const int i = own ? u : 0;
            float isyn = 0.0f;
            if (PAIR) isyn = row_current_pair(it, i, vcur[i], own);
            if (!own) continue;
            const float V = vcur[i];
            const VPre pre = neuron_v_pre(sg, i, N, V, ysc, y0, ylo, acc, prm, iext[i]);
            if (!PAIR) isyn = row_current<HAS2>(it, i, V);
            const float vn = neuron_v_post(sg, i, pre, isyn, y0, ylo, acc);
            vnxt[i] = vn;
            if (LAST && rec_slot >= 0) v.rec[rec_slot * v.N + lo + i] = vn;
        } else {
            const int p = u - nw;
            if (PAIR) {
                // gate of an own used pair for the next stage (same operations as
                // the per-synapse path), published in the other table
                const int t = __ldg(g.tix + (size_t)lo * nt + p);
                if (t < 0) continue;
                float2 f1;
                float4 f2 = make_float4(0.f, 0.f, 0.f, 0.f), d4 = f2;
                float4 &c2 = HAS2 ? cur2[p] : d4;
                float4 &a2 = HAS2 ? acc2[p] : d4;
                const float *sp = stab + (p % nt) * 9;
                coef_update<HAS2>(sp, vcur[p / nt], sg, cur1[p], acc1[p], f1, c2, a2, f2);
                const bool sec = HAS2 && sp[SP_KIND] != 0.0f;
                float G;
                if (!LAST) {
                    G = pair_gate(sec, cur1[p], c2, r0p[p], s0p[p], r0lo[p], s0lo[p]);
                } else {
                    // the step's end gates: the next step's first-stage gates and step-start state
                    float r0 = r0p[p], s0 = s0p[p], rl = r0lo[p], sl = s0lo[p];
                    pair_step(sec, f1, f2, r0, s0, rl, sl);
                    G = pair_gate(sec, make_float2(0.0f, 0.0f), make_float4(0.0f, 0.0f, 0.0f, f2.w), r0, s0, rl, sl);
                    r0p[p] = r0;
                    s0p[p] = s0;
                    r0lo[p] = rl;
                    s0lo[p] = sl;
                }
                gout[t] = G;
            } else {
                // gate map of an own pair: local copy for the next stage, and the
                // table every CTA reads at the next stage
                float2 f1;
                float4 f2 = make_float4(0.f, 0.f, 0.f, 0.f), d4 = f2;
                float4 &c2 = HAS2 ? cur2[p] : d4;
                float4 &a2 = HAS2 ? acc2[p] : d4;
                coef_update<HAS2>(stab + (p % nt) * 9, vcur[p / nt], sg, cur1[p], acc1[p], f1, c2, a2, f2);
                o1[p] = LAST ? f1 : cur1[p];
                if (HAS2) o2[p] = LAST ? f2 : cur2[p];
            }
        }
    }
    tgt = grid_arrive(g.bar);
    if (more) {
        // the next stage's gates of the owned neurons (own data only) while
        // the other CTAs arrive; that stage reads this one's ysn and vnxt
        // (after a step's last stage comes the first stage of the next step)
        float *ysx = ys + par * 3 * N;
        for (int i = nthr - 1 - tid; i < N; i += nthr) neuron_gates(sx, i, N, vnxt[i], ysn, ysx, y0, ylo, acc);
    }
    return true;
}

template <bool HAS2, bool PAIR>
__device__ void grid_run(const NetView &v, const GridView &g, long long step0, int nsteps, unsigned char *smem,
                         const float *stab) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int lo = g.row_split[blockIdx.x], N = g.row_split[blockIdx.x + 1] - lo;
    const int nt = v.n_stypes, Mloc = N * nt;
    const int M = (int)(v.N * nt);
    const NeuronLayout L = make_nlayout(N, N, Mloc, HAS2, PAIR, 0);  // the gate table sits after the layout
    float *y0 = (float *)(smem + L.y0), *ylo = (float *)(smem + L.ylo), *ys = (float *)(smem + L.ys);
    float *acc = (float *)(smem + L.acc);
    float *prm = (float *)(smem + L.prm), *iext = (float *)(smem + L.iext), *inp = (float *)(smem + L.inp);
    float *vst = (float *)(smem + L.vst);
    float2 *cur1 = (float2 *)(smem + L.cur1), *acc1 = (float2 *)(smem + L.acc1);
    float4 *cur2 = HAS2 ? (float4 *)(smem + L.cur2) : nullptr;
    float4 *acc2 = HAS2 ? (float4 *)(smem + L.acc2) : nullptr;
    int *tmp = (int *)(smem + L.tmp);
    float *pst = PAIR ? (float *)(smem + L.pair) : nullptr;
    float *gtab = PAIR ? (float *)(smem + L.syn) : nullptr;
    const int items1 = g.items[blockIdx.x], items2 = g.items[gridDim.x + blockIdx.x];
    Items it = PAIR ? carve_items_pair(smem + L.syn + 4LL * g.mt, N, g.K, items1)
                    : carve_items(smem + L.syn, N, g.K, items1, items2, HAS2);

    float *gV = v.state + lo;
    float *gr = v.state + 4 * v.N;
    float *gs = v.state + 4 * v.N + v.S;
    // the state's remainders (compensated sums), if the handle keeps them
    float *gVl = v.state_lo ? v.state_lo + lo : nullptr;
    float *grl = v.state_lo ? v.state_lo + 4 * v.N : nullptr;
    float *gsl = v.state_lo ? v.state_lo + 4 * v.N + v.S : nullptr;
    const bool keep_lo = gVl && g.r0lg;

    for (int i = tid; i < N; i += nthr) {
        const float V = gV[i];
        vst[i] = V;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const float y = gV[(long long)x * v.N + i];
            y0[x * N + i] = y;
            ylo[x * N + i] = gVl ? gVl[(long long)x * v.N + i] : 0.0f;
            if (x > 0) ys[(x - 1) * N + i] = y;  // stage-0 gates, parity 0
        }
        const float *p = v.nparams + (long long)v.neuron_type[lo + i] * PSST_NEURON_NPARAM;
        prm[NP_C * N + i] = 1.0f / p[NP_C];
#pragma unroll
        for (int x = 1; x < PSST_NEURON_NPARAM; ++x) prm[x * N + i] = p[x];
        inp[i] = v.i_const[lo + i];
        inp[N + i] = v.pulse_amp ? v.pulse_amp[lo + i] : 0.0f;
    }
    const long long pon = v.pulse_on[0], poff = v.pulse_off[0];
    if (PAIR) {
        // own pairs' step-start gates from one synapse of each, and their
        // stage-0 gates (identity step-end map) in table 0
        float *r0p = pst, *s0p = pst + Mloc, *r0lo = pst + 2 * Mloc, *s0lo = pst + 3 * Mloc;
        for (int p = tid; p < Mloc; p += nthr) {
            const int t = g.tix[(size_t)lo * nt + p];
            float r0 = 0.0f, s0 = 0.0f, rl = 0.0f, sl = 0.0f;
            if (t >= 0) {
                const float *sp = stab + (p % nt) * 9;
                const bool sec = HAS2 && sp[SP_KIND] != 0.0f;
                const long long k = g.rep[t];
                r0 = gr[k];
                if (sec) s0 = gs[k];
                if (keep_lo) {
                    rl = grl[k];
                    if (sec) sl = gsl[k];
                }
                g.gt[t] = pair_gate(sec, make_float2(0.0f, 0.0f),
                                    make_float4(0.0f, 0.0f, 0.0f, sec ? sp[SP_KD] : 1.0f), r0, s0, rl, sl);
            }
            r0p[p] = r0;
            s0p[p] = s0;
            r0lo[p] = rl;
            s0lo[p] = sl;
        }
        load_items_pair(it, v, 0, 0, lo, v.weight, v.syn_code, stab, tmp, g.tix);
    } else {
        // identity step-end maps of the own pairs in table 0 (read by stage 0)
        for (int p = tid; p < Mloc; p += nthr) {
            const int gi = lo * nt + p;
            g.c1[gi] = make_float2(0.0f, 0.0f);  // identity maps (increment form)
            if (HAS2) {
                const float *sp = stab + (p % nt) * 9;
                g.c2[gi] = make_float4(0.0f, 0.0f, 0.0f, sp[SP_KIND] != 0.0f ? sp[SP_KD] : 1.0f);
            }
        }
        load_items<HAS2>(it, v, 0, 0, lo, gr, gs, v.weight, v.syn_code, stab, tmp);
    }
    const float dt = v.dt;
    const int ns = method_stages(v);
    unsigned long long tgt = grid_arrive(g.bar);
    // the first stage's gates (own data) while the other CTAs finish setting up
    {
        const float *ysc = ys, *vcur = vst;
        float *ysn = ys + 3 * N;
        if (nsteps > 0) {
            const StageRT s0 = stage_rt(v, 0, dt);
            for (int i = nthr - 1 - tid; i < N; i += nthr) neuron_gates(s0, i, N, vcur[i], ysc, ysn, y0, ylo, acc);
        }
    }
    bool ok = true;
    // record: phase of (step + 1) modulo the stride, advanced once per step
    int rec_phase = v.rec_stride > 0 ? (int)((step0 + 1) % v.rec_stride) : -1;
    for (int itn = 0; ok && itn < nsteps; ++itn) {
        const long long step = step0 + itn;
        const bool in_pulse = step >= pon && step < poff;
        long long rec_slot = -1;
        if (rec_phase >= 0) {
            if (rec_phase == 0) rec_slot = ((step + 1) / v.rec_stride - 1) % v.rec_cap;
            rec_phase = rec_phase + 1 == v.rec_stride ? 0 : rec_phase + 1;
        }
        for (int i = tid; i < N; i += nthr)
            iext[i] = input_current(v, inp[i], inp[N + i], in_pulse, (long long)lo + i, step);
        const bool more = itn + 1 < nsteps;
        // stage s of step itn reads parity (itn * ns + s) & 1
#pragma unroll 1
        for (int s = 0; ok && s < ns; ++s) {
            const StageRT sg = stage_rt(v, s, dt), sx = stage_rt(v, s + 1 < ns ? s + 1 : 0, dt);
            ok = grid_stage<HAS2, PAIR>(v, g, sg, sx, it, lo, N, nt, M, rec_slot, vst, y0, ylo, acc, ys, prm, iext,
                                        cur1, acc1, cur2, acc2, pst, gtab, stab, (itn * ns + s) & 1, tgt,
                                        s + 1 < ns || more);
        }
        // the next step's input currents (own data) run before stage 0's wait
    }
    // the last stage's (or the setup's) barrier
    if (ok) ok = grid_wait(g.bar, tgt, g.timeout_ns, v.err);
    if (!ok) return;  // error recorded; global state keeps its value from before the call

    if (PAIR) {
        // the owners hand their pairs' gates to the CTAs owning the synapses
        const float *r0p = pst, *s0p = pst + Mloc, *r0lo = pst + 2 * Mloc, *s0lo = pst + 3 * Mloc;
        for (int p = tid; p < Mloc; p += nthr) {
            const int t = g.tix[(size_t)lo * nt + p];
            if (t >= 0) {
                g.r0g[t] = r0p[p];
                g.s0g[t] = s0p[p];
                if (keep_lo) {
                    g.r0lg[t] = r0lo[p];
                    g.s0lg[t] = s0lo[p];
                }
            }
        }
        if (!grid_barrier(g.bar, g.timeout_ns, v.err)) return;
        const long long k0 = v.row_ptr[lo], k1 = v.row_ptr[lo + N];
        for (long long k = k0 + tid; k < k1; k += nthr) {
            const uint32_t code = v.syn_code[k];
            const int t = g.tix[code & 0xFFFFFFu];
            const bool sec = HAS2 && second_order(stab, code);
            gr[k] = __ldcg(g.r0g + t);
            if (sec) gs[k] = __ldcg(g.s0g + t);
            if (keep_lo) {
                grl[k] = __ldcg(g.r0lg + t);
                if (sec) gsl[k] = __ldcg(g.s0lg + t);
            }
        }
    } else {
        // the last stage wrote the step's final maps into the table of the
        // launch's stage count's parity (RK4: four stages per step, table 0)
        const size_t fin = (size_t)(((long long)nsteps * ns) & 1);
        store_items<HAS2>(it, v, 0, 0, lo, gr, gs, v.syn_code, stab,
                          GlobalCoef{g.c1 + fin * M, HAS2 ? g.c2 + fin * M : nullptr});
    }
    bool bad = false;
    for (int i = tid; i < N; i += nthr) {
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const float y = y0[x * N + i];
            bad |= !isfinite(y);
            gV[(long long)x * v.N + i] = y;
            if (gVl) gVl[(long long)x * v.N + i] = ylo[x * N + i];
        }
    }
    if (bad) set_error(v.err, PSST_ERR_NONFINITE);
}

__global__ void __launch_bounds__(1024, 1) grid_kernel(NetView v, GridView g, long long step0, int nsteps) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float stab[PSST_MAX_SYN_TYPES * PSST_SYN_NPARAM];
    for (int i = threadIdx.x; i < v.n_stypes * PSST_SYN_NPARAM; i += blockDim.x) {
        float x = v.sparams[i];
        if (i % PSST_SYN_NPARAM == SP_KP) x = 1.0f / x;
        stab[i] = x;
    }
    __syncthreads();
    const bool has2 = v.net_flags[0] & NET_HAS2;
    if (g.pair) {
        if (has2) grid_run<true, true>(v, g, step0, nsteps, smem, stab);
        else grid_run<false, true>(v, g, step0, nsteps, smem, stab);
    } else {
        if (has2) grid_run<true, false>(v, g, step0, nsteps, smem, stab);
        else grid_run<false, false>(v, g, step0, nsteps, smem, stab);
    }
}

}  // namespace

cudaError_t grid_occupancy(int block, int smem, int *blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(grid_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, grid_kernel, block, smem);
}

cudaError_t grid_launch(const NetView &v, const GridView &g, long long step0, int nsteps, int grid, int block,
                        int smem, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(g.bar, 0, 2 * sizeof(unsigned), stream);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&v, (void *)&g, (void *)&step0, (void *)&nsteps};
    return cudaLaunchCooperativeKernel((const void *)grid_kernel, dim3(grid), dim3(block), args, (size_t)smem,
                                       stream);
}

}  // namespace psst
