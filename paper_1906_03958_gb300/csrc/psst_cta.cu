// Network-resident RK4 (or Euler) integration for batches of small and
// medium networks.
//
// One network is owned by a cluster of CL CTAs (CL = 1, 2 or 4, chosen per
// network by its shared-memory footprint) for all of a launch's steps.  Each
// CTA of the cluster owns a block of rows (postsynaptic neurons): their
// synapses, as work items in shared memory (psst_syn.cuh), and their neuron
// state.  Every CTA keeps the stage potential of all N neurons and the gate
// maps of all used (neuron, type) pairs.  One launch per size class
// integrates all networks of that class, largest first; the classes run on
// their own streams.  Networks without synapses are integrated elsewhere
// (psst_indep.cu).
//
// Per RK4 step (classic tableau, Sec. "Brain simulations as computational
// graphs", RK4 paragraph) and stage s = 0..3 (Euler: one stage; a given
// tableau: its 1..4 stages):
//   S-phase   each thread sums its work items (per-pair layout: A = sum w G
//             with the pair's gate G gathered from the gate table), after
//             the owned neurons' gates m, h, n (on the highest threads);
//   barrier   (CTA);
//   N-phase   one work loop over independent units: the potential of each
//             owned neuron (its row's item partials give I_syn, then the HH
//             currents and the stage update; the next stage potential goes
//             to every CTA of the cluster through distributed shared
//             memory), and the gate map (and per-pair gate) of every entry
//             from the stage-s potentials (identical values in every CTA);
//             the potentials take whole warps;
//   barrier   CTA barrier (CL = 1) or cluster barrier (CL > 1).
// Stage potentials and gates are double-buffered by parity, so a CTA can
// write the next stage's values while a peer still reads this stage's.
//
// Synaptic gates: a gate's equation dr/dt = a T_j (1 - r) - b r is affine in
// r with coefficients set by its presynaptic neuron j alone, so each RK4
// stage value is r^(s) = P_s[j] + Q_s[j] r0 (second-order pairs:
// s^(s) = U_s + X_s r0 + Z_s s0) with the maps propagated once per
// (neuron, type) and stage; the step-end map is applied lazily at the next
// step's first stage.  This evaluates the same RK4 map as the textbook stage
// recursion.  When all gates of a pair are equal (from rest) one gate per
// pair is kept (per-pair layout); else each synapse applies the map to its
// own gate with one FMA per stage.
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

// One stage sg of the handle's method: a compile-time descriptor (the four
// classic RK4 stages, StageCT) or a run-time one (StageRT: one copy of this
// code serves every stage of Euler and of a tableau); both give the same
// bits.  par selects the double-buffered stage potentials and gates read by
// this stage: the parity of the stage's index counted over the launch.
template <int CL, bool HAS2, bool PAIR, class SG>
__device__ __forceinline__ void stage(const NetView &v, const SG &sg, const Items &it, int n0, int N, int nt,
                                      int M, int r_lo, int nown, unsigned rank, long long rec_slot, float *vst,
                                      float *y0, float *ylo, float *acc, float *ys, const float *prm,
                                      const float *iext,
                                      float2 *cur1, float2 *acc1, float2 *fin1, float4 *cur2, float4 *acc2,
                                      float4 *fin2, float *pst, float *Gt, int lrep, const float *stab, int par) {
    const bool FIRST = sg.first, LAST = sg.last;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const float *vcur = vst + par * N;
    float *vnxt = vst + (par ^ 1) * N;
    const float *ysc = ys + par * 3 * nown;
    float *ysn = ys + (par ^ 1) * 3 * nown;
    // gate-map entries: every (neuron, type) pair, or the used pairs (PAIR)
    float *r0p = pst, *s0p = pst + M, *r0lo = pst + 2 * M, *s0lo = pst + 3 * M;
    const unsigned *pof = (const unsigned *)(pst + 4 * M);  // per-pair entries: neuron << 8 | type
    // The gates m, h, n of the owned neurons need only this stage's
    // potentials: they are computed before the S-phase (on the highest
    // threads), where their latency overlaps the S-phase's loads, and leave
    // the N-phase fewer units.
    for (int i = nthr - 1 - tid; i < nown; i += nthr)
        neuron_gates(sg, i, nown, vcur[r_lo + i], ysc, ysn, y0, ylo, acc);
    if (PAIR) sphase_pair(it, Gt, lrep);
    else sphase<HAS2>(FIRST, it, SmemCoef{FIRST ? fin1 : cur1, FIRST ? fin2 : cur2});
    __syncthreads();
    // independent work units: potential of each owned neuron and the gate
    // map (and per-pair gate) of each entry; the potentials take whole warps
    const int nw = (nown + 31) & ~31;
    const int U = nw + M;
    for (int u = tid; u < U; u += nthr) {
        if (u < nw) {
            // the whole warp takes this branch (nw and nthr are multiples of 32)
            const bool own = u < nown;
            const int i = own ? u : 0;
            float isyn = 0.0f;
            if (PAIR) isyn = row_current_pair(it, i, vcur[r_lo + i], own);
            if (!own) continue;
            const float V = vcur[r_lo + i];
            const VPre pre = neuron_v_pre(sg, i, nown, V, ysc, y0, ylo, acc, prm, iext[i]);
            if (!PAIR) isyn = row_current<HAS2>(it, i, V);
            const float vn = neuron_v_post(sg, i, pre, isyn, y0, ylo, acc);
            vnxt[r_lo + i] = vn;
            if (CL > 1) {
#pragma unroll
                for (unsigned q = 1; q < CL; ++q) st_peer(vnxt + r_lo + i, (rank + q) % CL, vn);
            }
            if (LAST && rec_slot >= 0) v.rec[rec_slot * v.N + n0 + r_lo + i] = vn;
        } else {
            const int p = u - nw;
            float4 d4 = make_float4(0.f, 0.f, 0.f, 0.f);
            float4 &c2 = HAS2 ? cur2[p] : d4;
            float4 &a2 = HAS2 ? acc2[p] : d4;
            float4 &f2 = HAS2 ? fin2[p] : d4;
            // presynaptic neuron and synapse type of the entry
            const int pre = PAIR ? (int)(pof[p] >> 8) : p / nt, tp = PAIR ? (int)(pof[p] & 255u) : p % nt;
            const float *sp = stab + tp * 9;
            coef_update<HAS2>(sp, vcur[pre], sg, cur1[p], acc1[p], fin1[p], c2, a2, f2);
            if (PAIR) {
                // the pair's gate for the next stage (same operations as the per-synapse path)
                const bool sec = HAS2 && sp[SP_KIND] != 0.0f;
                if (!LAST) {
                    put_gate(Gt, p, lrep, pair_gate(sec, cur1[p], c2, r0p[p], s0p[p], r0lo[p], s0lo[p]));
                } else {
                    // the step's end gates: the next step's first-stage gates and step-start state
                    float r0 = r0p[p], s0 = s0p[p], rl = r0lo[p], sl = s0lo[p];
                    pair_step(sec, fin1[p], f2, r0, s0, rl, sl);
                    put_gate(Gt, p, lrep, pair_gate(sec, make_float2(0.0f, 0.0f), make_float4(0.0f, 0.0f, 0.0f, f2.w),
                                                    r0, s0, rl, sl));
                    r0p[p] = r0;
                    s0p[p] = s0;
                    r0lo[p] = rl;
                    s0lo[p] = sl;
                }
            }
        }
    }
    if (CL > 1) cluster_sync();
    else __syncthreads();
}

template <int CL, bool HAS2, bool PAIR>
__device__ void run_net(const NetView &v, int b, const NetPlan &pl, long long step0, int nsteps, int lrep_cap,
                        unsigned char *smem, const float *stab) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const unsigned rank = CL > 1 ? cluster_rank() : 0u;
    const int n0 = v.net_off[b], N = v.net_off[b + 1] - n0;
    const int nt = v.n_stypes;
    // gate-map entries: all (neuron, type) pairs, or the network's used pairs
    const int M = PAIR ? v.pair_off[b + 1] - v.pair_off[b] : N * nt;
    const int *ptix = PAIR ? v.pair_tix + (long long)n0 * nt : nullptr;  // local pair -> entry
    const long long sbase = v.row_ptr[n0];
    const int r_lo = pl.split[rank], nown = pl.split[rank + 1] - r_lo;
    const int lrep = PAIR ? min(pl.lrep, lrep_cap) : 0;  // copies of the gate table (at most the plan's)
    const NeuronLayout L = make_nlayout(nown, N, M, HAS2, PAIR, 1 << lrep);
    float *y0 = (float *)(smem + L.y0), *ylo = (float *)(smem + L.ylo), *ys = (float *)(smem + L.ys);
    float *acc = (float *)(smem + L.acc);
    float *prm = (float *)(smem + L.prm), *iext = (float *)(smem + L.iext), *inp = (float *)(smem + L.inp);
    float *vst = (float *)(smem + L.vst);
    float2 *cur1 = (float2 *)(smem + L.cur1), *acc1 = (float2 *)(smem + L.acc1), *fin1 = (float2 *)(smem + L.fin1);
    float4 *cur2 = HAS2 ? (float4 *)(smem + L.cur2) : nullptr;
    float4 *acc2 = HAS2 ? (float4 *)(smem + L.acc2) : nullptr;
    float4 *fin2 = HAS2 ? (float4 *)(smem + L.fin2) : nullptr;
    int *tmp = (int *)(smem + L.tmp);
    float *pst = PAIR ? (float *)(smem + L.pair) : nullptr;
    float *Gt = PAIR ? (float *)(smem + L.gt) : nullptr;
    Items it = PAIR ? carve_items_pair(smem + L.syn, nown, pl.K, pl.n1[rank])
                    : carve_items(smem + L.syn, nown, pl.K, pl.n1[rank], pl.n2[rank], HAS2);

    float *gV = v.state + n0;
    float *gr = v.state + 4 * v.N + sbase;
    float *gs = v.state + 4 * v.N + v.S + sbase;
    // the state's remainders (compensated sums), if the handle keeps them
    float *gVl = v.state_lo ? v.state_lo + n0 : nullptr;
    float *grl = v.state_lo ? v.state_lo + 4 * v.N + sbase : nullptr;
    float *gsl = v.state_lo ? v.state_lo + 4 * v.N + v.S + sbase : nullptr;
    const float *gw = v.weight + sbase;
    const uint32_t *gcode = v.syn_code + sbase;

    for (int j = tid; j < N; j += nthr) vst[j] = gV[j];  // stage-0 potentials, parity 0
    for (int i = tid; i < nown; i += nthr) {
        const int gi = r_lo + i;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const float y = gV[(long long)x * v.N + gi];
            y0[x * nown + i] = y;
            ylo[x * nown + i] = gVl ? gVl[(long long)x * v.N + gi] : 0.0f;
            if (x > 0) ys[(x - 1) * nown + i] = y;  // stage-0 gates, parity 0
        }
        const float *p = v.nparams + (long long)v.neuron_type[n0 + gi] * PSST_NEURON_NPARAM;
        prm[NP_C * nown + i] = 1.0f / p[NP_C];
#pragma unroll
        for (int x = 1; x < PSST_NEURON_NPARAM; ++x) prm[x * nown + i] = p[x];
        inp[i] = v.i_const[n0 + gi];
        inp[nown + i] = v.pulse_amp ? v.pulse_amp[n0 + gi] : 0.0f;
    }
    const long long pon = v.pulse_on[b], poff = v.pulse_off[b];
    unsigned *pof = PAIR ? (unsigned *)(pst + 4 * M) : nullptr;
    if (PAIR)
        for (int k = tid; k < M; k += nthr) {
            const int ci = v.pair_of[v.pair_off[b] + k];  // local pair: neuron * nt + type
            pof[k] = ((unsigned)(ci / nt) << 8) | (unsigned)(ci % nt);
        }
    for (int k = tid; k < M; k += nthr) {
        fin1[k] = make_float2(0.0f, 0.0f);  // identity maps (increment form)
        if (HAS2) {
            const int ci = PAIR ? v.pair_of[v.pair_off[b] + k] : k;
            const float *sp = stab + (ci % nt) * 9;
            fin2[k] = make_float4(0.0f, 0.0f, 0.0f, sp[SP_KIND] != 0.0f ? sp[SP_KD] : 1.0f);
        }
    }
    if (PAIR) {
        // pair state from the network's synapses (all gates of a pair are equal)
        for (int p = tid; p < 4 * M; p += nthr) pst[p] = 0.0f;
        __syncthreads();
        const int S = (int)(v.row_ptr[n0 + N] - sbase);
        for (int k = tid; k < S; k += nthr) {
            const int t = ptix[gcode[k] & 0xFFFFFFu];
            const bool sec = HAS2 && second_order(stab, gcode[k]);
            pst[t] = gr[k];
            if (sec) pst[M + t] = gs[k];
            if (grl) {
                pst[2 * M + t] = grl[k];
                if (sec) pst[3 * M + t] = gsl[k];
            }
        }
        __syncthreads();
        for (int p = tid; p < M; p += nthr) {
            const bool sec = HAS2 && stab[(pof[p] & 255u) * 9 + SP_KIND] != 0.0f;
            put_gate(Gt, p, lrep,
                     pair_gate(sec, fin1[p], HAS2 ? fin2[p] : make_float4(0.f, 0.f, 0.f, 1.f), pst[p], pst[M + p],
                               pst[2 * M + p], pst[3 * M + p]));
        }
        load_items_pair(it, v, n0, sbase, r_lo, gw, gcode, stab, tmp, ptix);  // ends with __syncthreads
    } else {
        load_items<HAS2>(it, v, n0, sbase, r_lo, gr, gs, gw, gcode, stab, tmp);  // ends with __syncthreads
    }
    if (CL > 1) cluster_sync();

    const float dt = v.dt;
    const int ns = method_stages(v);
    // record: phase of (step + 1) modulo the stride, advanced once per step
    int rec_phase = v.rec_stride > 0 ? (int)((step0 + 1) % v.rec_stride) : -1;
    for (int itn = 0; itn < nsteps; ++itn) {
        const long long step = step0 + itn;
        const bool in_pulse = step >= pon && step < poff;
        long long rec_slot = -1;
        if (rec_phase >= 0) {
            if (rec_phase == 0) rec_slot = ((step + 1) / v.rec_stride - 1) % v.rec_cap;
            rec_phase = rec_phase + 1 == v.rec_stride ? 0 : rec_phase + 1;
        }
        for (int i = tid; i < nown; i += nthr)
            iext[i] = input_current(v, inp[i], inp[nown + i], in_pulse, (long long)n0 + r_lo + i, step);
        // iext is read in the N-phase, after the S-phase barrier
        // stage s of step itn reads parity (itn * ns + s) & 1
#define PSST_STAGE(SG, par)                                                                                    \
    stage<CL, HAS2, PAIR>(v, SG, it, n0, N, nt, M, r_lo, nown, rank, rec_slot, vst, y0, ylo, acc, ys, prm, iext, \
                          cur1, acc1, fin1, cur2, acc2, fin2, pst, Gt, lrep, stab, par)
        if (v.method == PSST_METHOD_RK4) {
            // the classic tableau's stages at compile time (no stage-kind branches on the hot path)
            PSST_STAGE(StageCT<0>{stage_coef<0>(v, dt)}, 0);
            PSST_STAGE(StageCT<1>{stage_coef<1>(v, dt)}, 1);
            PSST_STAGE(StageCT<2>{stage_coef<2>(v, dt)}, 0);
            PSST_STAGE(StageCT<3>{stage_coef<3>(v, dt)}, 1);
        } else {
#pragma unroll 1
            for (int s = 0; s < ns; ++s) PSST_STAGE(stage_rt(v, s, dt), (itn * ns + s) & 1);
        }
#undef PSST_STAGE
    }

    // write back: owned synapses with the last step's gate map, owned neurons
    if (PAIR) {
        const long long k0 = v.row_ptr[n0 + r_lo] - sbase, k1 = v.row_ptr[n0 + r_lo + nown] - sbase;
        for (long long k = k0 + tid; k < k1; k += nthr) {
            const int t = ptix[gcode[k] & 0xFFFFFFu];
            const bool sec = HAS2 && second_order(stab, gcode[k]);
            gr[k] = pst[t];
            if (sec) gs[k] = pst[M + t];
            if (grl) {
                grl[k] = pst[2 * M + t];
                if (sec) gsl[k] = pst[3 * M + t];
            }
        }
    } else {
        store_items<HAS2>(it, v, n0, sbase, r_lo, gr, gs, gcode, stab, SmemCoef{fin1, fin2});
    }
    bool bad = false;
    for (int i = tid; i < nown; i += nthr) {
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const float y = y0[x * nown + i];
            bad |= !isfinite(y);
            gV[(long long)x * v.N + r_lo + i] = y;
            if (gVl) gVl[(long long)x * v.N + r_lo + i] = ylo[x * nown + i];
        }
    }
    if (bad) set_error(v.err, PSST_ERR_NONFINITE);
    if (CL > 1) cluster_sync();  // no CTA leaves while a peer may still write into it
}

template <int CL>
__global__ void __launch_bounds__(1024) net_kernel(NetView v, const int *list, const NetPlan *plans,
                                                   long long step0, int nsteps, int lrep_cap) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float stab[PSST_MAX_SYN_TYPES * PSST_SYN_NPARAM];
    for (int i = threadIdx.x; i < v.n_stypes * PSST_SYN_NPARAM; i += blockDim.x) {
        float x = v.sparams[i];
        if (i % PSST_SYN_NPARAM == SP_KP) x = 1.0f / x;  // stored as 1/Kp
        stab[i] = x;
    }
    __syncthreads();
    const int b = list[blockIdx.x / CL];
    const uint8_t f = v.net_flags[b];
    if (f & NET_PAIR) {
        if (f & NET_HAS2) run_net<CL, true, true>(v, b, plans[b], step0, nsteps, lrep_cap, smem, stab);
        else run_net<CL, false, true>(v, b, plans[b], step0, nsteps, lrep_cap, smem, stab);
    } else {
        if (f & NET_HAS2) run_net<CL, true, false>(v, b, plans[b], step0, nsteps, lrep_cap, smem, stab);
        else run_net<CL, false, false>(v, b, plans[b], step0, nsteps, lrep_cap, smem, stab);
    }
}

template <int CL>
cudaError_t launch_cl(const NetView &v, const ClassLaunch &c, long long step0, int nsteps, cudaStream_t stream) {
    if (CL == 1) {
        net_kernel<1><<<c.n_nets, c.block, c.smem, stream>>>(v, c.list, c.plans, step0, nsteps, c.lrep_cap);
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
    return cudaLaunchKernelEx(&cfg, net_kernel<CL>, v, c.list, c.plans, step0, nsteps, c.lrep_cap);
}

// out[b] = 1 when every (presynaptic neuron, type) pair of network b has
// bitwise-equal gates (r, s) in the state; one CTA per network, shared
// memory holds the first synapse of each pair.
__global__ void pair_check_kernel(NetView v, uint8_t *out) {
    extern __shared__ int first[];
    __shared__ int bad;
    const int b = blockIdx.x, tid = threadIdx.x, nthr = blockDim.x;
    const int n0 = v.net_off[b], N = v.net_off[b + 1] - n0, M = N * v.n_stypes;
    const long long sbase = v.row_ptr[n0], S = v.row_ptr[n0 + N] - sbase;
    const uint32_t *code = v.syn_code + sbase;
    const float *r = v.state + 4 * v.N + sbase, *s = v.state + 4 * v.N + v.S + sbase;
    for (int p = tid; p < M; p += nthr) first[p] = 0x7fffffff;
    if (tid == 0) bad = 0;
    __syncthreads();
    for (long long k = tid; k < S; k += nthr) atomicMin(&first[code[k] & 0xFFFFFFu], (int)k);
    __syncthreads();
    for (long long k = tid; k < S; k += nthr) {
        const int f = first[code[k] & 0xFFFFFFu];
        if (__float_as_uint(r[k]) != __float_as_uint(r[f]) || __float_as_uint(s[k]) != __float_as_uint(s[f])) bad = 1;
    }
    __syncthreads();
    if (tid == 0) out[b] = bad ? 0 : 1;
}

}  // namespace

cudaError_t pair_check(const NetView &v, uint8_t *out, int smem, cudaStream_t stream) {
    cudaError_t e = cudaFuncSetAttribute(pair_check_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    pair_check_kernel<<<v.n_nets, 256, smem, stream>>>(v, out);
    return cudaGetLastError();
}

int cta_static_smem() { return (int)(PSST_MAX_SYN_TYPES * PSST_SYN_NPARAM * sizeof(float)); }

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
