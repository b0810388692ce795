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
// table through L2; one device-wide synchronisation per RK4 stage separates
// writers from readers, and double buffering removes the write-after-read
// hazard.
//
// Per-pair variant (all gates of each (presynaptic neuron, type) pair equal,
// as from rest): the owner of a presynaptic neuron keeps its pairs' gate
// state and publishes each used pair's next-stage gate as one 8-byte word,
// the stage's phase number in the high half and the gate value in the low
// half, written by a single 64-bit store.  A reader accepts a word when its
// tag shows the phase it waits for, so every word carries its own "ready"
// and no fence or flag sits between writer and reader: each CTA copies the
// whole table into shared memory as the words arrive and gathers its
// synapses' gates from there, instead of gathering an 8-byte map per
// synapse from L2.  Each CTA also writes one tagged heartbeat word per
// stage, after its own copy of the previous table, so that a CTA which has
// seen every word of a phase knows that every CTA is done reading the
// buffer it is about to overwrite (double buffering, as for the maps).
// Both buffers are zeroed before each launch (phases start at 1).  Results
// are bitwise equal to the per-synapse variant.
//
// The per-synapse variant reads its maps straight from L2 during the
// S-phase; there each CTA publishes the phase it has finished in a flag of
// its own (a release: fence, then a relaxed store) and waits by polling
// every flag (acquire loads).  The step-end hand-off of the per-pair
// variant uses the same flags.  Waits are bounded: on expiry a CTA records
// PSST_ERR_TIMEOUT and every CTA returns.
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

__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long *p) {
    unsigned long long x;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(x) : "l"(p) : "memory");
    return x;
}

// The same load without a compiler memory barrier, for the self-checking
// words of the gate table (their order against other accesses is free).
__device__ __forceinline__ unsigned long long ld_relaxed64_word(const unsigned long long *p) {
    unsigned long long x;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(x) : "l"(p));
    return x;
}

__device__ __forceinline__ void st_relaxed64(unsigned long long *p, unsigned long long x) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(x) : "memory");
}

__device__ __forceinline__ void fence_acq_rel_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

// grid_publish: the CTA has finished phase `phase` (numbered 1, 2, ... over
// the launch); after all its threads' global writes of the phase.  Each
// CTA's flag has a 128-byte line of its own, so that the polls of
// different flags go to different L2 slices.
__device__ __forceinline__ void grid_publish(const GridView &g, unsigned long long phase) {
    __syncthreads();
    if (threadIdx.x == 0) {
        fence_acq_rel_gpu();  // with the store: a release of the CTA's writes
        st_relaxed64(g.flag + (size_t)blockIdx.x * GRID_FLAG_STRIDE, phase);
    }
}

// grid_gather: wait until every CTA has published `phase` (flags).  Warp w
// polls the flags of CTAs w, w + nwarps, ... (up to 32 at a time, lane j
// the j-th, all in one acquire load per round) until all have shown it.
// Returns false (after recording the error) when a wait ran out of time or
// another CTA already failed.
__device__ bool grid_gather(const GridView &g, unsigned long long phase, int *err, int *s_fail) {
    const int G = gridDim.x, lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    bool fail = false;
    for (int base = warp; base < G && !fail; base += 32 * nwarp) {
        const int mine = base + lane * nwarp;  // this lane's flag
        const unsigned long long *f = g.flag + (size_t)(mine < G ? mine : 0) * GRID_FLAG_STRIDE;
        unsigned pending = __ballot_sync(0xffffffffu, mine < G);
        unsigned long long t0 = 0;
        while (pending) {
            const bool up = ((pending >> lane) & 1u) && ld_acquire64(f) >= phase;
            const unsigned seen = __ballot_sync(0xffffffffu, up);
            pending &= ~seen;
            if (seen || !pending) continue;
            const unsigned long long now = globaltimer();
            if (t0 == 0) t0 = now;
            if (__any_sync(0xffffffffu, *(volatile int *)err != 0)) {
                fail = true;
                break;
            }
            if (__any_sync(0xffffffffu, now - t0 > g.timeout_ns)) {
                if (lane == 0) set_error(err, PSST_ERR_TIMEOUT);
                fail = true;
                break;
            }
        }
    }
    if (fail) *s_fail = 1;
    __syncthreads();
    return *(volatile int *)s_fail == 0;
}

// A gate-table word: phase tag (high half), value (low half).  Tags are
// the phase modulo 2^32; a word read for phase q was last written for
// phase q - 2 (or zeroed), so the wrap never makes a stale word match.
__device__ __forceinline__ unsigned long long gate_word(unsigned long long phase, float G) {
    return ((unsigned long long)(unsigned)phase << 32) | __float_as_uint(G);
}

constexpr int GT_BATCH = 8;  // table words a thread loads before it checks them

// grid_gather_table: copy the values of the words [0, used) of the tagged
// table src into dst (shared memory), and check the heartbeat words
// [used, used + gridDim.x), once each shows `phase`.  Thread t takes words
// t, t + blockDim.x, ..., loading GT_BATCH of them before checking any;
// a word with an older tag is read again until it shows the phase (bounded
// wait, as grid_gather).
__device__ bool grid_gather_table(const GridView &g, unsigned long long phase, const unsigned long long *src,
                                  float *dst, int *err, int *s_fail) {
    const int used = g.used, nw = used + gridDim.x, nthr = blockDim.x;
    const unsigned tag = (unsigned)phase;
    bool fail = false;
    for (int e0 = threadIdx.x; e0 < nw && !fail; e0 += GT_BATCH * nthr) {
        unsigned long long w[GT_BATCH];
#pragma unroll
        for (int b = 0; b < GT_BATCH; ++b) {
            const int e = e0 + b * nthr;
            w[b] = e < nw ? ld_relaxed64_word(src + e) : gate_word(phase, 0.0f);
        }
#pragma unroll
        for (int b = 0; b < GT_BATCH; ++b) {
            const int e = e0 + b * nthr;
            unsigned long long x = w[b];
            if ((unsigned)(x >> 32) != tag) {
                const unsigned long long t0 = globaltimer();
                while ((unsigned)((x = ld_relaxed64_word(src + e)) >> 32) != tag) {
                    if (*(volatile int *)err != 0) {
                        fail = true;
                        break;
                    }
                    if (globaltimer() - t0 > g.timeout_ns) {
                        set_error(err, PSST_ERR_TIMEOUT);
                        fail = true;
                        break;
                    }
                }
                if (fail) break;
            }
            if (e < used) dst[e] = __uint_as_float((unsigned)x);
        }
    }
    if (fail) *s_fail = 1;
    __syncthreads();
    return *(volatile int *)s_fail == 0;
}

struct GlobalCoef {
    const float2 *t1;
    const float4 *t2;
    __device__ __forceinline__ float2 r(int i) const { return __ldcg(t1 + i); }
    __device__ __forceinline__ float4 s(int i) const { return __ldcg(t2 + i); }
};

// One stage sg of the handle's method (a compile-time StageCT for the
// classic RK4 stages, else a run-time StageRT: one copy of this code serves
// every stage of Euler and a tableau); sx is the stage after it;
// par selects the double-buffered potentials, gates and global tables this
// stage reads (the parity of the stage's index counted over the launch).  On
// entry the owned neurons' gates m, h, n of this stage are done and `phase`
// is the phase every CTA must have published; on return the CTA has
// published the next phase (phase updated) and, when `more`, computed the
// next stage's (sx's) gates.
template <bool HAS2, bool PAIR, class SG, class SX>
__device__ __forceinline__ bool grid_stage(const NetView &v, const GridView &g, const SG &sg, const SX &sx,
                                           const Items &it, int lo, int N, int nt, int M,
                                           long long rec_slot, float *vst, float *y0, float *ylo, float *acc,
                                           float *ys,
                                           const float *prm, const float *iext, float2 *cur1, float2 *acc1,
                                           float4 *cur2, float4 *acc2, float *pst, float *gtab, const float *stab,
                                           int par, unsigned long long &phase, bool more, int *s_fail) {
    const bool LAST = sg.last;
    const int tid = threadIdx.x, nthr = blockDim.x, Mloc = N * nt;
    const float *vcur = vst + par * N;
    float *vnxt = vst + (par ^ 1) * N;
    const float *ysc = ys + par * 3 * N;
    float *ysn = ys + (par ^ 1) * 3 * N;
    // the other CTAs' gates and maps of this stage are published (per pair:
    // this stage's gate of every used pair, copied as each owner's flag shows it)
    if (PAIR) {
        if (!grid_gather_table(g, phase, g.gt + (size_t)par * g.gts, gtab, v.err, s_fail)) return false;
        sphase_pair(it, gtab, 0);
    } else {
        if (!grid_gather(g, phase, v.err, s_fail)) return false;
        sphase<HAS2>(sg.first, it, GlobalCoef{g.c1 + (size_t)par * M, HAS2 ? g.c2 + (size_t)par * M : nullptr});
    }
    __syncthreads();
    // independent work units: potential of each owned neuron and the gate map
    // of each own (neuron, type) pair; the potentials take whole warps
    float *r0p = pst, *s0p = pst + Mloc, *r0lo = pst + 2 * Mloc, *s0lo = pst + 3 * Mloc;
    unsigned long long *gout = PAIR ? g.gt + (size_t)(par ^ 1) * g.gts : nullptr;
    // this CTA is done reading the other table: its heartbeat for the next phase
    if (PAIR && tid == 0) st_relaxed64(gout + g.used + blockIdx.x, gate_word(phase + 1, 0.0f));
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
                st_relaxed64(gout + t, gate_word(phase + 1, G));
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
    if (PAIR) {
        __syncthreads();  // the next stage's gates read this stage's potentials
        ++phase;
    } else {
        grid_publish(g, ++phase);
    }
    if (more) {
        // the next stage's gates of the owned neurons (own data only) while
        // the other CTAs finish; that stage reads this one's ysn and vnxt
        // (after a step's last stage comes the first stage of the next step)
        float *ysx = ys + par * 3 * N;
        for (int i = nthr - 1 - tid; i < N; i += nthr) neuron_gates(sx, i, N, vnxt[i], ysn, ysx, y0, ylo, acc);
    }
    return true;
}

template <bool HAS2, bool PAIR>
__device__ void grid_run(const NetView &v, const GridView &g, long long step0, int nsteps, unsigned char *smem,
                         const float *stab, int *s_fail) {
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
                const float G0 = pair_gate(sec, make_float2(0.0f, 0.0f),
                                           make_float4(0.0f, 0.0f, 0.0f, sec ? sp[SP_KD] : 1.0f), r0, s0, rl, sl);
                st_relaxed64(g.gt + t, gate_word(1, G0));
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
    // phase 1: the setup's writes (tagged table words and heartbeats, or the
    // identity maps behind a flag)
    unsigned long long phase = 1;
    if (PAIR) {
        if (tid == 0) st_relaxed64(g.gt + g.used + blockIdx.x, gate_word(1, 0.0f));
        __syncthreads();
    } else {
        grid_publish(g, phase);
    }
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
#define PSST_GSTAGE(SG, SX, par, mo)                                                                            \
    grid_stage<HAS2, PAIR>(v, g, SG, SX, it, lo, N, nt, M, rec_slot, vst, y0, ylo, acc, ys, prm, iext, cur1, acc1, \
                           cur2, acc2, pst, gtab, stab, par, phase, mo, s_fail)
        if (v.method == PSST_METHOD_RK4) {
            const StageCT<0> k0{stage_coef<0>(v, dt)};
            const StageCT<1> k1{stage_coef<1>(v, dt)};
            const StageCT<2> k2{stage_coef<2>(v, dt)};
            const StageCT<3> k3{stage_coef<3>(v, dt)};
            ok = PSST_GSTAGE(k0, k1, 0, true);
            if (ok) ok = PSST_GSTAGE(k1, k2, 1, true);
            if (ok) ok = PSST_GSTAGE(k2, k3, 0, true);
            if (ok) ok = PSST_GSTAGE(k3, k0, 1, more);
        } else {
#pragma unroll 1
            for (int s = 0; ok && s < ns; ++s) {
                const StageRT sg = stage_rt(v, s, dt), sx = stage_rt(v, s + 1 < ns ? s + 1 : 0, dt);
                ok = PSST_GSTAGE(sg, sx, (itn * ns + s) & 1, s + 1 < ns || more);
            }
        }
#undef PSST_GSTAGE
        // the next step's input currents (own data) run before stage 0's wait
    }
    // the last stage's (or the setup's) phase
    if (ok && !PAIR) ok = grid_gather(g, phase, v.err, s_fail);
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
        grid_publish(g, ++phase);
        if (!grid_gather(g, phase, v.err, s_fail)) return;
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
    __shared__ int s_fail;  // set by any thread whose wait failed
    if (threadIdx.x == 0) s_fail = 0;
    for (int i = threadIdx.x; i < v.n_stypes * PSST_SYN_NPARAM; i += blockDim.x) {
        float x = v.sparams[i];
        if (i % PSST_SYN_NPARAM == SP_KP) x = 1.0f / x;
        stab[i] = x;
    }
    __syncthreads();
    const bool has2 = v.net_flags[0] & NET_HAS2;
    if (g.pair) {
        if (has2) grid_run<true, true>(v, g, step0, nsteps, smem, stab, &s_fail);
        else grid_run<false, true>(v, g, step0, nsteps, smem, stab, &s_fail);
    } else {
        if (has2) grid_run<true, false>(v, g, step0, nsteps, smem, stab, &s_fail);
        else grid_run<false, false>(v, g, step0, nsteps, smem, stab, &s_fail);
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
    cudaError_t e = cudaMemsetAsync(g.flag, 0, (size_t)grid * GRID_FLAG_STRIDE * sizeof(unsigned long long), stream);
    if (e == cudaSuccess && g.pair) e = cudaMemsetAsync(g.gt, 0, 2 * (size_t)g.gts * sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return e;
    void *args[] = {(void *)&v, (void *)&g, (void *)&step0, (void *)&nsteps};
    return cudaLaunchCooperativeKernel((const void *)grid_kernel, dim3(grid), dim3(block), args, (size_t)smem,
                                       stream);
}

}  // namespace psst
