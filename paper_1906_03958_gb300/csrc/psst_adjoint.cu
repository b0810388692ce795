// Discrete adjoint of the RK4 or forward-Euler network map (the
// differentiated form).
//
// Gradient of L = sum_f sum_i dL/dV[f][i] V_i(frame f) over n steps from
// the current state, with respect to every synaptic weight and every
// neuron-type parameter, for batches of networks (one cluster of two CTAs per
// network: one recomputes segments forward, the other sweeps them backward).
//
// Gate state.  When all gates of a (presynaptic neuron j, synapse type tau)
// pair start from the same value -- as they do from rest -- they stay equal
// for ever, since their equation depends only on V_j and the type.  The
// kernel then carries one gate (r, and s for second order) per pair: the
// same trajectory as the per-synapse model, with state 4N + 2M
// (M = N * n_types) instead of 4N + 2S.  psst_adjoint checks the
// precondition on the starting state.
//
// Reverse sweep (Hager 2000; Sandu 2006).  For the step y_n -> y_{n+1} with
// stages Y_s and k_s = f(Y_s):
//   kb4 = h/6 lam,           Yb4 = J(Y4)^T kb4
//   kb3 = h/3 lam + h Yb4,   Yb3 = J(Y3)^T kb3
//   kb2 = h/3 lam + h/2 Yb3, Yb2 = J(Y2)^T kb2
//   kb1 = h/6 lam + h/2 Yb2, Yb1 = J(Y1)^T kb1
//   lam_n = lam + Yb1 + Yb2 + Yb3 + Yb4;  theta_bar += sum_s (df/dtheta)^T kb_s.
// Forward Euler (Eq. euler) is the one-stage case: kb1 = h lam,
// lam_n = lam + J(y_n)^T kb1.  A tableau (stage s starts at
// y + h a_s k_{s-1}, weights b_s) has kb_s = h b_s lam + h a_{s+1} Yb_{s+1}.
// The forward kernel records the full state and its compensated-sum
// remainders every `ckpt` steps (psst_integrate with recording, run by
// psst_adjoint itself when the caller recorded nothing); each segment is
// recomputed forward from its checkpoint, keeping every step's stages in
// global memory, then swept backward from those stages.  The recomputation
// carries the remainders too (compensated state, psst_device.cuh).
//
// Jacobian-transpose product at a stage (q_i = kbV_i / C_i,
// A_i = sum_k w_k G_p(k), G_p the pair's gate, I_syn = V A - B):
//   uV_i = q_i (-dI_ion/dV - A_i) + sum_x kbx_i (alpha_x' (1-x) - beta_x' x)
//          + sum_tau kbr_(i,tau) a T'(V_i) (1 - r_(i,tau))
//   um_i = -q_i 3 gNa m^2 h (V - ENa) - kbm_i (alpha_m + beta_m), likewise h, n
//   ur_p = -C_p [first order] - (a T + b) kbr_p + K3 kbs_p [second order]
//   us_p = -C_p G'(s_p) - K4 kbs_p               [second order]
//   with the column sum C_p = sum_{k in p} w_k (q_i V_i - q_i E_k);
//   dL/dw_k += -q_i G_p (V_i - E_k);  dL/dgNa += -q_i m^3 h (V - ENa), ...
// The two CTAs hold the synapses in different layouts: the forward CTA
// in row items (the synaptic current's row sums), the sweeping CTA in
// column items, the synapses of each pair p cut into items of KC chunks of
// 4 with the column's m-th synapse (rows in CSR order) in item m mod nq,
// position m / nq (nq = the pair's items), so that the lanes of a warp
// gather the stage products (q_i V_i, q_i) of consecutive rows.  One
// thread per column item sums w (q_i V_i - E_p q_i) over its synapses;
// the pair's owner adds its items' partials in item order (fixed order,
// reproducible).  The weight gradients are summed over each step's stages
// in one pass over the column items, into an FP32 partial per segment,
// then into an FP64 total.  Per stage the sweep runs its per-neuron work as
// independent units on separate threads: part A (the potential's products
// and parameter gradients; each gate variable's rates, its adjoint and its
// term of uV), the column sums, part C (each pair's adjoints and its term of
// uV; then each neuron adds its terms in a fixed order).  The parameter
// gradients are compensated FP32 sums, combined in FP64 at the end.
#include <cuda_runtime.h>

#include "psst_device.cuh"
#include "psst_internal.h"

namespace psst {

namespace {

constexpr int ADJ_THREADS = 1024;

__device__ __forceinline__ unsigned cluster_rank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

// Barrier of the cluster's CTAs; release/acquire orders their global memory
// accesses across it.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ float ratio_u_deriv(float u) {
    // d/du of u / (1 - e^{-u}); Bernoulli series near 0
    if (fabsf(u) < 0.1f) {
        const float u2 = u * u;
        return fmaf(u, fmaf(u2, -1.0f / 180.0f, 1.0f / 6.0f), 0.5f);
    }
    const float e = expf(-u), den = -expm1f(-u);
    return __fdiv_rn(den - u * e, den * den);
}

struct AdjSmem {
    // forward CTA: row items (row-aligned, K chunks of 4 synapses,
    // slot-major) with the pair of each synapse in id; sweeping CTA: column
    // items (KC chunks, slot-major) with the row of each synapse in id
    float4 *w;
    ushort4 *id;
    float *pa, *pb;    // forward: item partials A and B; sweep: column item partials (pa)
    int *ib;           // forward: [N+1] first item of each row; sweep: [M+1] first item of each pair
    unsigned short *irow;  // sweep: [n_citems] pair of each column item
    // per stage s = 0..3 (stored by the forward recompute)
    float *sV, *sm, *sh, *sn;  // [4][N]
    float *sr, *ss, *sG;       // [4][M]
    float *sA, *sfv;           // [4][N]
    // reduced state y (step start) and running RK4 sums
    float *y;                  // [4N + 2M]: V, m, h, n, r, s
    float *ylo;                // [4N + 2M]: remainders of y (compensated step sums)
    float *acc;                // [4N + 2M]
    // adjoint
    float *lam, *yprev, *ysum; // [4N + 2M]
    float2 *ab;                // [4][N]: q_i V_i, q_i at each stage
    float *uV;                 // [N] partial uV
    float2 *gp;                // [N][9] neuron parameter gradients, compensated FP32 sums (hi, lo)
    float2 *uvc;               // [M] each pair's term of its presynaptic potential's adjoint
    float2 *uvg;               // [3][N] each gate's term of its neuron's potential adjoint (kb, derivative)
    float *Ep;                 // [M] reversal potential of each pair's type
    float *prm;                // [9][N] (row 0: 1/C)
    float *iext, *inp;         // [N], [2][N]
};

// Row items of the forward CTA (K chunks each) and column items of the
// sweeping CTA (KC chunks each) share one region of shared memory.
__host__ __device__ inline long long adj_item_chunks(int n_items, int K, int n_citems, int KC) {
    const long long r = (long long)K * n_items, c = (long long)KC * n_citems;
    return r > c ? r : c;
}

__host__ __device__ inline long long adj_smem_bytes(int N, int M, int n_items, int K, int n_citems, int KC) {
    long long b = 0;
    const long long chunks = adj_item_chunks(n_items, K, n_citems, KC);
    const long long parts = 8LL * n_items > 4LL * n_citems ? 8LL * n_items : 4LL * n_citems;
    b += chunks * (16 + 8);             // w, id
    b += parts + 2LL * n_citems + 16;   // pa, pb (column partials), irow
    b += 4LL * ((N > M ? N : M) + 1);   // ib
    b += 4LL * 4 * (6LL * N + 3LL * M);  // stage storage
    b += 4LL * 6 * (4LL * N + 2LL * M);  // y, ylo, acc, lam, yprev, ysum
    b += 32LL * N + 4LL * N;             // ab, uV
    b += 8LL * 9 * N;                    // gp (float2)
    b += 8LL * M;                        // uvc
    b += 24LL * N;                       // uvg
    b += 4LL * 9 * N + 4LL * 3 * N;      // prm, iext, inp
    b += 4LL * M;                        // Ep
    b += 16 * 32;                        // alignment slack
    return b;
}

__device__ inline unsigned char *take(unsigned char *&p, long long bytes) {
    unsigned char *at = p;
    p += (bytes + 15) & ~15LL;
    return at;
}

struct AdjNet {
    int b, n0, N, nt, M, K, n_items, KC, n_citems, R;
    long long sbase, S;
};

// ---------------------------------------------------------------- forward

// Forward of one step of the reduced model from S.y (step `step`) with NST
// stages (4: RK4, 1: forward Euler; TAB: the handle's tableau of NST
// stages), storing the stages' values; on return S.y holds the next state.
template <bool STORE, int NST, bool TAB>
__device__ void fwd_step(const NetView &v, const AdjNet &a, const AdjSmem &S, const float *stab, long long step,
                         float dt) {
    const int tid = threadIdx.x, nthr = blockDim.x, N = a.N, nt = a.nt, M = a.M;
    float *V = S.y, *m = S.y + N, *h = S.y + 2 * N, *n = S.y + 3 * N, *r = S.y + 4 * N, *s = S.y + 4 * N + M;
    const bool in_pulse = step >= v.pulse_on[a.b] && step < v.pulse_off[a.b];
    for (int i = tid; i < N; i += nthr)
        S.iext[i] = input_current(v, S.inp[i], S.inp[N + i], in_pulse, (long long)a.n0 + i, step);
    // stage values live in the stage arrays (stage 0 = y)
    for (int i = tid; i < N; i += nthr) {
        S.sV[i] = V[i];
        S.sm[i] = m[i];
        S.sh[i] = h[i];
        S.sn[i] = n[i];
        for (int t = 0; t < nt; ++t) {
            const int p = i * nt + t;
            const float *sp = stab + t * 9;
            S.sr[p] = r[p];
            S.ss[p] = s[p];
            const float s2 = s[p] * s[p], s4 = s2 * s2;
            S.sG[p] = sp[SP_KIND] != 0.0f ? __fdiv_rn(s4, s4 + sp[SP_KD]) : r[p];
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int st = 0; st < NST; ++st) {
        const float *G = S.sG + st * M;
        // synaptic sums per item
        const int K = a.K, ni = a.n_items;
        for (int it = tid; it < ni; it += nthr) {
            float A = 0.0f, B = 0.0f;
            for (int j = 0; j < K; ++j) {
                const int c = j * ni + it;
                const float4 w = S.w[c];
                const ushort4 id = S.id[c];
                const float g0 = G[id.x], g1 = G[id.y], g2 = G[id.z], g3 = G[id.w];
                A = fmaf(w.x, g0, A);
                A = fmaf(w.y, g1, A);
                A = fmaf(w.z, g2, A);
                A = fmaf(w.w, g3, A);
                B = fmaf(w.x * S.Ep[id.x], g0, B);
                B = fmaf(w.y * S.Ep[id.y], g1, B);
                B = fmaf(w.z * S.Ep[id.z], g2, B);
                B = fmaf(w.w * S.Ep[id.w], g3, B);
            }
            S.pa[it] = A;
            S.pb[it] = B;
        }
        __syncthreads();
        const float WGT = TAB ? v.rk_w[st] : (st == 0 || st == 3) ? 1.0f : 2.0f;
        const float cnext = TAB ? (st < 3 ? v.rk_c[st] * dt : 0.0f) : (st == 2) ? dt : 0.5f * dt;
        const float dt6 = TAB ? v.rk_beta * dt : NST == 1 ? dt : dt * (1.0f / 6.0f);  // scale of the step's sum
        const float W0 = TAB ? v.rk_w[0] : 1.0f;  // weight of the first stage's slope
        // independent units, each on its own thread: the potential of each
        // neuron (row sums, ionic current), its gates m, h, n (rate
        // functions) and every gate pair (transmitter, r and s)
        float *stg[4] = {S.sV, S.sm, S.sh, S.sn};
        for (int u = tid; u < 2 * N + M; u += nthr) {
            if (u < N) {
                const int i = u;
                float A = 0.0f, B = 0.0f;
                for (int it = S.ib[i]; it < S.ib[i + 1]; ++it) {
                    A += S.pa[it];
                    B += S.pb[it];
                }
                const float Vs = S.sV[st * N + i], ms = S.sm[st * N + i], hs = S.sh[st * N + i],
                            ns = S.sn[st * N + i];
                const float *P = S.prm;
                const float m3h = ms * ms * ms * hs, n4 = ns * ns * ns * ns;
                const float iion = P[NP_GNA * N + i] * m3h * (Vs - P[NP_ENA * N + i]) +
                                   P[NP_GK * N + i] * n4 * (Vs - P[NP_EK * N + i]) +
                                   P[NP_GL * N + i] * (Vs - P[NP_EL * N + i]) +
                                   P[NP_GKL * N + i] * (Vs - P[NP_EKL * N + i]);
                const float fV = (S.iext[i] - iion - fmaf(Vs, A, -B)) * P[NP_C * N + i];
                if (STORE) {
                    S.sA[st * N + i] = A;
                    S.sfv[st * N + i] = fV;
                }
                const float ac = (st == 0) ? W0 * fV : fmaf(WGT, fV, S.acc[i]);
                if (st < NST - 1) {
                    S.acc[i] = ac;
                    S.sV[(st + 1) * N + i] = ext_stage(S.y[i], S.ylo[i], cnext, fV);
                } else {
                    ext_step(S.y[i], S.ylo[i], dt6, ac);
                }
            } else if (u < 2 * N) {
                const int i = u - N;
                const float Vs = S.sV[st * N + i], ms = S.sm[st * N + i], hs = S.sh[st * N + i],
                            ns = S.sn[st * N + i];
                const Rates q = hh_rates(Vs);
                const float d[3] = {q.am * (1.0f - ms) - q.bm * ms, q.ah * (1.0f - hs) - q.bh * hs,
                                    q.an * (1.0f - ns) - q.bn * ns};
#pragma unroll
                for (int x = 1; x < 4; ++x) {
                    const int ix = x * N + i;
                    const float ac = (st == 0) ? W0 * d[x - 1] : fmaf(WGT, d[x - 1], S.acc[ix]);
                    if (st < NST - 1) {
                        S.acc[ix] = ac;
                        stg[x][(st + 1) * N + i] = ext_stage(S.y[ix], S.ylo[ix], cnext, d[x - 1]);
                    } else {
                        ext_step(S.y[ix], S.ylo[ix], dt6, ac);
                    }
                }
            } else {
                // gate pair p = (presynaptic neuron i, type t)
                const int p = u - 2 * N, i = p / nt, t = p - i * nt;
                const float *sp = stab + t * 9;
                const float Vs = S.sV[st * N + i];
                const float rs = S.sr[st * M + p], ss = S.ss[st * M + p];
                const float T = transmitter(Vs, sp[SP_VP], sp[SP_KP]);
                const float dr = sp[SP_A] * T * (1.0f - rs) - sp[SP_B] * rs;
                const float ds = sp[SP_KIND] != 0.0f ? sp[SP_K3] * rs - sp[SP_K4] * ss : 0.0f;
                const int ir = 4 * N + p, is = 4 * N + M + p;
                const float ar = (st == 0) ? W0 * dr : fmaf(WGT, dr, S.acc[ir]);
                const float as = (st == 0) ? W0 * ds : fmaf(WGT, ds, S.acc[is]);
                if (st < NST - 1) {
                    S.acc[ir] = ar;
                    S.acc[is] = as;
                    const float rn = ext_stage(S.y[ir], S.ylo[ir], cnext, dr);
                    const float sn = ext_stage(S.y[is], S.ylo[is], cnext, ds);
                    S.sr[(st + 1) * M + p] = rn;
                    S.ss[(st + 1) * M + p] = sn;
                    const float s2 = sn * sn, s4 = s2 * s2;
                    S.sG[(st + 1) * M + p] = sp[SP_KIND] != 0.0f ? __fdiv_rn(s4, s4 + sp[SP_KD]) : rn;
                } else {
                    ext_step(S.y[ir], S.ylo[ir], dt6, ar);
                    ext_step(S.y[is], S.ylo[is], dt6, as);
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- reverse

// Column sums of stage st: each column item's partial
// sum_k w_k (q_i V_i - E_p q_i) over its synapses in slot order, into S.pa.
__device__ __forceinline__ void column_sums(const AdjNet &a, const AdjSmem &S, int st) {
    const int tid = threadIdx.x, nthr = blockDim.x, KC = a.KC, nc = a.n_citems;
    const float2 *ab = S.ab + st * a.N;
    for (int t = tid; t < nc; t += nthr) {
        const float E = S.Ep[S.irow[t]];
        float c = 0.0f;
#pragma unroll 4
        for (int j = 0; j < KC; ++j) {
            const int q = j * nc + t;
            const float4 w = S.w[q];
            const ushort4 r = S.id[q];
            const float2 a0 = ab[r.x], a1 = ab[r.y], a2 = ab[r.z], a3 = ab[r.w];
            c = fmaf(w.x, fmaf(-E, a0.y, a0.x), c);
            c = fmaf(w.y, fmaf(-E, a1.y, a1.x), c);
            c = fmaf(w.z, fmaf(-E, a2.y, a2.x), c);
            c = fmaf(w.w, fmaf(-E, a3.y, a3.x), c);
        }
        S.pa[t] = c;
    }
}

// Reverse of the step whose NST stages fwd_step<true, NST, .> just stored:
// lam holds the adjoint of y_{n+1} on entry and of y_n on exit (before the
// frame term).  cb[s] = h b_s, ca[s] = h a_{s+1} (the factor of stage s's
// slope in stage s+1's start).
template <int NST>
__device__ void rev_step(const AdjNet &a, const AdjSmem &S, const float *stab, const float *cb, const float *ca,
                         float4 *gpart) {
    const int tid = threadIdx.x, nthr = blockDim.x, N = a.N, nt = a.nt, M = a.M;
#pragma unroll 1
    for (int st = NST - 1; st >= 0; --st) {
        // A) four units per neuron: the potential's products (ab, the base of
        // uV) and parameter gradients, and one per gate variable (its term of
        // uV, kept for part C, and its adjoint); whole warps per unit kind
        const int Nw = (N + 31) & ~31;
        for (int u = tid; u < 4 * Nw; u += nthr) {
            const int x = u / Nw, i = u - x * Nw;  // x = 0: potential, 1..3: gate m, h, n
            if (i >= N) continue;
            const bool gates = x > 0;
            const float Vs = S.sV[st * N + i], ms = S.sm[st * N + i], hs = S.sh[st * N + i], ns = S.sn[st * N + i];
            const float *P = S.prm;
            const float kb0 = cb[st] * S.lam[i] + (st < NST - 1 ? ca[st] * S.yprev[i] : 0.0f);
            const float q = kb0 * P[NP_C * N + i];
            const float m3h = ms * ms * ms * hs, n4 = ns * ns * ns * ns;
            const float gNa = P[NP_GNA * N + i], gK = P[NP_GK * N + i], gL = P[NP_GL * N + i], gKL = P[NP_GKL * N + i];
            const float ENa = P[NP_ENA * N + i], EK = P[NP_EK * N + i];
            if (!gates) {
                const float EL = P[NP_EL * N + i], EKL = P[NP_EKL * N + i];
                S.ab[st * N + i] = make_float2(q * Vs, q);
                const float diion = gNa * m3h + gK * n4 + gL + gKL;
                S.uV[i] = q * (-diion - S.sA[st * N + i]);
                // compensated FP32 sums (hi, lo) of the stage terms
                float2 *g = S.gp + 9 * i;
                auto add = [&](int x, float term) {
                    float2 c = g[x];
                    ext_add(c.x, c.y, term);
                    g[x] = c;
                };
                add(NP_C, -q * S.sfv[st * N + i]);
                add(NP_GNA, -q * m3h * (Vs - ENa));
                add(NP_GK, -q * n4 * (Vs - EK));
                add(NP_GL, -q * (Vs - EL));
                add(NP_GKL, -q * (Vs - EKL));
                add(NP_ENA, q * gNa * m3h);
                add(NP_EK, q * gK * n4);
                add(NP_EL, q * gL);
                add(NP_EKL, q * gKL);
            } else {
                // gate x: its rate functions (those of hh_rates) and their derivatives
                const int ix = x * N + i;
                const float kbx = cb[st] * S.lam[ix] + (st < NST - 1 ? ca[st] * S.yprev[ix] : 0.0f);
                float al, be, dal, dbe, g, yp;
                if (x == 1) {
                    al = ratio_u((Vs + 40.0f) * 0.1f);
                    be = 4.0f * expf((Vs + 65.0f) * (-1.0f / 18.0f));
                    dal = 0.1f * ratio_u_deriv((Vs + 40.0f) * 0.1f);
                    dbe = -be * (1.0f / 18.0f);
                    g = ms;
                    yp = -q * gNa * 3.0f * ms * ms * hs * (Vs - ENa);
                } else if (x == 2) {
                    al = 0.07f * expf((Vs + 65.0f) * (-1.0f / 20.0f));
                    be = __frcp_rn(1.0f + expf((Vs + 35.0f) * (-0.1f)));
                    dal = -al * (1.0f / 20.0f);
                    dbe = be * (1.0f - be) * 0.1f;
                    g = hs;
                    yp = -q * gNa * ms * ms * ms * (Vs - ENa);
                } else {
                    al = 0.1f * ratio_u((Vs + 55.0f) * 0.1f);
                    be = 0.125f * expf((Vs + 65.0f) * (-1.0f / 80.0f));
                    dal = 0.01f * ratio_u_deriv((Vs + 55.0f) * 0.1f);
                    dbe = -be * (1.0f / 80.0f);
                    g = ns;
                    yp = -q * gK * 4.0f * ns * ns * ns * (Vs - EK);
                }
                S.uvg[(x - 1) * N + i] = make_float2(kbx, dal * (1.0f - g) - dbe * g);
                S.yprev[ix] = yp - kbx * (al + be);
            }
        }
        __syncthreads();
        // B) column sums of the synaptic current's Jacobian
        column_sums(a, S, st);
        __syncthreads();
        // C) one unit per gate pair (its adjoints and its term of the
        // presynaptic potential's adjoint), then one per neuron (the terms in
        // type order)
        for (int p = tid; p < M; p += nthr) {
            const int i = p / nt, t = p - i * nt;
            const float Vs = S.sV[st * N + i];
            const float *sp = stab + t * 9;
            float C = 0.0f;  // the pair's column sum: its items' partials in item order
            for (int q = S.ib[p]; q < S.ib[p + 1]; ++q) C += S.pa[q];
            const int ir = 4 * N + p, is = 4 * N + M + p;
            const float kbr = cb[st] * S.lam[ir] + (st < NST - 1 ? ca[st] * S.yprev[ir] : 0.0f);
            const float kbs = cb[st] * S.lam[is] + (st < NST - 1 ? ca[st] * S.yprev[is] : 0.0f);
            const float rs = S.sr[st * M + p], ss = S.ss[st * M + p];
            const float T = transmitter(Vs, sp[SP_VP], sp[SP_KP]);
            const float dT = T * (1.0f - T) * sp[SP_KP];  // table holds 1/Kp
            float ur = -(sp[SP_A] * T + sp[SP_B]) * kbr, us = 0.0f;
            if (sp[SP_KIND] != 0.0f) {
                const float s2 = ss * ss, s4 = s2 * s2, den = s4 + sp[SP_KD];
                const float dG = __fdiv_rn(4.0f * s2 * ss * sp[SP_KD], den * den);
                ur = fmaf(sp[SP_K3], kbs, ur);
                us = -C * dG - sp[SP_K4] * kbs;
            } else {
                ur -= C;
            }
            S.uvc[p] = make_float2(kbr * sp[SP_A] * dT, 1.0f - rs);
            S.yprev[ir] = ur;
            S.yprev[is] = us;
            S.ysum[ir] += ur;
            S.ysum[is] += us;
        }
        __syncthreads();
        for (int i = tid; i < N; i += nthr) {
            float uV = S.uV[i];
#pragma unroll
            for (int x = 0; x < 3; ++x) {
                const float2 c = S.uvg[x * N + i];
                uV = fmaf(c.x, c.y, uV);
            }
            for (int t = 0; t < nt; ++t) {
                const float2 c = S.uvc[i * nt + t];
                uV = fmaf(c.x, c.y, uV);
            }
            S.yprev[i] = uV;
            S.ysum[i] += uV;
            S.ysum[N + i] += S.yprev[N + i];
            S.ysum[2 * N + i] += S.yprev[2 * N + i];
            S.ysum[3 * N + i] += S.yprev[3 * N + i];
        }
        __syncthreads();  // the next stage's part A reads yprev of both units of each neuron
    }
    // weight gradients of the step: dL/dw_k += sum_s -G_p^(s) q_i^(s) (V_i^(s) - E_p),
    // into the per-segment FP32 partial of each column slot (the partials of
    // up to four chunks loaded before any is updated)
    const int KC = a.KC, nc = a.n_citems;
    for (int t = tid; t < nc; t += nthr) {
        const int p = S.irow[t];
        const float E = S.Ep[p];
        float G[NST];
#pragma unroll
        for (int st = 0; st < NST; ++st) G[st] = S.sG[st * M + p];
        for (int j0 = 0; j0 < KC; j0 += 4) {
            float4 g[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (j0 + u < KC) g[u] = gpart[(j0 + u) * nc + t];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (j0 + u >= KC) break;
                const int c = (j0 + u) * nc + t;
                const ushort4 r = S.id[c];
                const int iv[4] = {r.x, r.y, r.z, r.w};
                float gv[4] = {g[u].x, g[u].y, g[u].z, g[u].w};
#pragma unroll
                for (int q4 = 0; q4 < 4; ++q4) {
                    float acc = 0.0f;
#pragma unroll
                    for (int st = 0; st < NST; ++st) {
                        const float2 abv = S.ab[st * N + iv[q4]];
                        acc = fmaf(G[st], fmaf(E, abv.y, -abv.x), acc);
                    }
                    gv[q4] += acc;
                }
                gpart[c] = make_float4(gv[0], gv[1], gv[2], gv[3]);
            }
        }
    }
    // lam_n = lam + sum of the stage adjoints (owner-only values)
    for (int i = tid; i < N; i += nthr) {
        for (int x = 0; x < 4; ++x) {
            const int ix = x * N + i;
            S.lam[ix] += S.ysum[ix];
            S.ysum[ix] = 0.0f;
        }
        for (int t = 0; t < nt; ++t) {
            const int ir = 4 * N + i * nt + t, is = 4 * N + M + i * nt + t;
            S.lam[ir] += S.ysum[ir];
            S.lam[is] += S.ysum[is];
            S.ysum[ir] = 0.0f;
            S.ysum[is] = 0.0f;
        }
    }
    __syncthreads();
}

// Reduced state of the network from a full state [V, m, h, n, r, s] of the
// whole batch and its remainders full_lo (null: zero): neurons as they are,
// each pair's gates from its synapses (all equal by the precondition; *bad,
// if given, is set when they differ).
__device__ void load_reduced(const NetView &v, const AdjNet &a, const AdjSmem &S, const float *full,
                             const float *full_lo, const long long *rp, const uint32_t *gcode, int *bad) {
    const int tid = threadIdx.x, nthr = blockDim.x, N = a.N, M = a.M;
    const float *gr = full + 4 * v.N + a.sbase, *gs = full + 4 * v.N + v.S + a.sbase;
    const float *grl = full_lo ? full_lo + 4 * v.N + a.sbase : nullptr;
    const float *gsl = full_lo ? full_lo + 4 * v.N + v.S + a.sbase : nullptr;
    for (int i = tid; i < N; i += nthr)
        for (int x = 0; x < 4; ++x) {
            S.y[x * N + i] = full[(long long)x * v.N + a.n0 + i];
            S.ylo[x * N + i] = full_lo ? full_lo[(long long)x * v.N + a.n0 + i] : 0.0f;
        }
    for (int q = tid; q < M; q += nthr) {
        S.y[4 * N + q] = 0.0f;
        S.y[4 * N + M + q] = 0.0f;
        S.ylo[4 * N + q] = 0.0f;
        S.ylo[4 * N + M + q] = 0.0f;
    }
    __syncthreads();
    for (int i = tid; i < N; i += nthr)
        for (long long k = rp[i] - a.sbase; k < rp[i + 1] - a.sbase; ++k) {
            const int ci = (int)(gcode[k] & 0xFFFFFFu);
            S.y[4 * N + ci] = gr[k];
            S.y[4 * N + M + ci] = gs[k];
            if (grl) {
                S.ylo[4 * N + ci] = grl[k];
                S.ylo[4 * N + M + ci] = gsl[k];
            }
        }
    __syncthreads();
    if (bad) {
        for (int i = tid; i < N; i += nthr)
            for (long long k = rp[i] - a.sbase; k < rp[i + 1] - a.sbase; ++k) {
                const int ci = (int)(gcode[k] & 0xFFFFFFu);
                if (S.y[4 * N + ci] != gr[k] || S.y[4 * N + M + ci] != gs[k]) *bad = 1;
            }
        __syncthreads();
    }
}

// Floats a step keeps in a segment buffer: the NST stages' values of V, m, h,
// n, A and f_V per neuron and r, s, G per pair.
__host__ __device__ inline long long adj_step_floats(int nst, long long N, long long M) {
    return (long long)nst * (6 * N + 3 * M);
}

// Copy of the first nst stages of the stage arrays (sV .. sfv, each
// [4][len], stage-major) to or from a compact block of nst (6N + 3M) floats
// (the step record of a method with fewer than four stages).
template <bool TO_BLOCK>
__device__ void copy_stages(float *stages, float *blk, int N, int M, int nst) {
    const int nN = nst * N, nM = nst * M, tot = 6 * nN + 3 * nM;
    for (int q = threadIdx.x; q < tot; q += blockDim.x) {
        int at;
        if (q < 4 * nN) {
            at = 4 * N * (q / nN) + q % nN;  // V, m, h, n
        } else if (q < 4 * nN + 3 * nM) {
            const int r = q - 4 * nN;
            at = 16 * N + 4 * M * (r / nM) + r % nM;  // r, s, G
        } else {
            const int r = q - 4 * nN - 3 * nM;
            at = 16 * N + 12 * M + 4 * N * (r / nN) + r % nN;  // A, f_V
        }
        if (TO_BLOCK) blk[q] = stages[at];
        else stages[at] = blk[q];
    }
}

template <int NST, bool TAB>
__global__ void __launch_bounds__(ADJ_THREADS) adj_kernel(NetView v, AdjView av, long long step0, int nsteps) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float stab[PSST_MAX_SYN_TYPES * PSST_SYN_NPARAM];
    __shared__ int s_bad;
    for (int i = threadIdx.x; i < v.n_stypes * PSST_SYN_NPARAM; i += blockDim.x) {
        float x = v.sparams[i];
        if (i % PSST_SYN_NPARAM == SP_KP) x = 1.0f / x;
        stab[i] = x;
    }
    if (threadIdx.x == 0) s_bad = 0;
    __syncthreads();
    const int tid = threadIdx.x, nthr = blockDim.x;
    AdjNet a;
    a.b = blockIdx.x / 2;  // one 2-CTA cluster per network
    a.n0 = v.net_off[a.b];
    a.N = v.net_off[a.b + 1] - a.n0;
    a.nt = v.n_stypes;
    a.M = a.N * a.nt;
    a.K = av.K[a.b];
    a.n_items = av.n_items[a.b];
    a.KC = av.KC[a.b];
    a.n_citems = av.n_citems[a.b];
    a.R = 4 * a.N + 2 * a.M;
    a.sbase = v.row_ptr[a.n0];
    a.S = v.row_ptr[a.n0 + a.N] - a.sbase;
    const int N = a.N, M = a.M, nt = a.nt, K = a.K, ni = a.n_items, nc = a.n_citems;
    // the two CTAs of the network's cluster: rank 0 recomputes segments
    // forward, rank 1 sweeps them backward and owns the gradients
    const bool fwd_cta = cluster_rank() == 0;

    AdjSmem S;
    unsigned char *p = smem;
    const long long chunks = adj_item_chunks(ni, K, nc, a.KC);
    S.w = (float4 *)take(p, 16 * chunks);
    S.id = (ushort4 *)take(p, 8 * chunks);
    S.pa = (float *)take(p, 8LL * ni > 4LL * nc ? 8LL * ni : 4LL * nc);
    S.pb = S.pa + ni;
    S.irow = (unsigned short *)take(p, 2LL * nc);
    S.ib = (int *)take(p, 4LL * ((N > M ? N : M) + 1));
    S.sV = (float *)take(p, 16LL * N);
    S.sm = (float *)take(p, 16LL * N);
    S.sh = (float *)take(p, 16LL * N);
    S.sn = (float *)take(p, 16LL * N);
    S.sr = (float *)take(p, 16LL * M);
    S.ss = (float *)take(p, 16LL * M);
    S.sG = (float *)take(p, 16LL * M);
    S.sA = (float *)take(p, 16LL * N);
    S.sfv = (float *)take(p, 16LL * N);
    S.y = (float *)take(p, 4LL * a.R);
    S.ylo = (float *)take(p, 4LL * a.R);
    S.acc = (float *)take(p, 4LL * a.R);
    S.lam = (float *)take(p, 4LL * a.R);
    S.yprev = (float *)take(p, 4LL * a.R);
    S.ysum = (float *)take(p, 4LL * a.R);
    S.ab = (float2 *)take(p, 32LL * N);
    S.uV = (float *)take(p, 4LL * N);
    S.gp = (float2 *)take(p, 72LL * N);
    S.uvc = (float2 *)take(p, 8LL * M);
    S.uvg = (float2 *)take(p, 24LL * N);
    S.Ep = (float *)take(p, 4LL * M);
    S.prm = (float *)take(p, 36LL * N);
    S.iext = (float *)take(p, 4LL * N);
    S.inp = (float *)take(p, 8LL * N);

    const long long *rp = v.row_ptr + a.n0;
    const uint32_t *gcode = v.syn_code + a.sbase;
    const float *gw = v.weight + a.sbase;

    // neurons, parameters, inputs; initial reduced state
    for (int i = tid; i < N; i += nthr) {
        const float *pp = v.nparams + (long long)v.neuron_type[a.n0 + i] * PSST_NEURON_NPARAM;
        S.prm[NP_C * N + i] = 1.0f / pp[NP_C];
        for (int x = 1; x < PSST_NEURON_NPARAM; ++x) S.prm[x * N + i] = pp[x];
        S.inp[i] = v.i_const[a.n0 + i];
        S.inp[N + i] = v.pulse_amp ? v.pulse_amp[a.n0 + i] : 0.0f;
        for (int x = 0; x < 9; ++x) S.gp[9 * i + x] = make_float2(0.0f, 0.0f);
        S.uV[i] = 0.0f;
    }
    for (int q = tid; q < M; q += nthr) S.Ep[q] = stab[(q % nt) * 9 + SP_E];
    for (int q = tid; q < a.R; q += nthr) {
        S.lam[q] = 0.0f;
        S.ysum[q] = 0.0f;
        S.yprev[q] = 0.0f;
    }
    float *W = (float *)S.w;
    unsigned short *ID = (unsigned short *)S.id;
    const long long cslot0 = av.cslot_off[a.b];
    if (fwd_cta) {
        // row items: row-aligned, each row's synapses in CSR order
        const long long slots = (long long)K * ni;
        int *cnt = (int *)S.acc;  // scratch: acc is written before it is read
        for (int i = tid; i < N; i += nthr) cnt[i] = (int)((rp[i + 1] - rp[i] + 4 * K - 1) / (4 * K));
        __syncthreads();
        if (tid == 0) {
            int acc = 0;
            for (int i = 0; i < N; ++i) {
                S.ib[i] = acc;
                acc += cnt[i];
            }
            S.ib[N] = acc;
        }
        for (long long c = tid; c < slots; c += nthr) {
            S.w[c] = make_float4(0.f, 0.f, 0.f, 0.f);
            S.id[c] = make_ushort4(0, 0, 0, 0);
        }
        __syncthreads();
        for (int i = tid; i < N; i += nthr) {
            const long long k0 = rp[i] - a.sbase;
            for (long long k = k0; k < rp[i + 1] - a.sbase; ++k) {
                const int m = (int)(k - k0);
                const int t = S.ib[i] + m / (4 * K), j = (m % (4 * K)) >> 2;
                const long long slot = ((long long)j * ni + t) * 4 + (m & 3);
                W[slot] = gw[k];
                ID[slot] = (unsigned short)(gcode[k] & 0xFFFFFFu);
            }
        }
    } else {
        // column items (host plan): the pair of each item, each slot's
        // synapse (-1: padding, w = 0) and row
        const int *cib = av.cib + av.cib_off[a.b];
        for (int q = tid; q <= M; q += nthr) S.ib[q] = cib[q];
        __syncthreads();
        for (int q = tid; q < M; q += nthr)
            for (int t = S.ib[q]; t < S.ib[q + 1]; ++t) S.irow[t] = (unsigned short)q;
        const int *ck = av.ck + cslot0;
        const unsigned short *cr = av.crow + cslot0;
        for (long long q = tid; q < 4LL * a.KC * nc; q += nthr) {
            const int k = ck[q];
            W[q] = k >= 0 ? gw[k] : 0.0f;
            ID[q] = cr[q];
        }
    }
    __syncthreads();
    // starting state (reduced; the span's first checkpoint), checked for
    // equal gates within each pair
    load_reduced(v, a, S, av.ck_full, av.ck_full_lo, rp, gcode, &s_bad);
    if (s_bad) {
        if (tid == 0) set_error(v.err, PSST_ERR_UNSUPPORTED);
        return;
    }

    // the stage arrays form one contiguous block (sV .. sfv) of stage_floats;
    // a step keeps step_floats of it (its NST stages)
    const int stage_floats = 4 * (6 * N + 3 * M);
    const int step_floats = (int)adj_step_floats(NST, N, M);
    float4 *stage_blk = (float4 *)S.sV;
    const int ckpt = av.ckpt_every;
    const float dt = v.dt;
    // h b_s and h a_{s+1} of the method (RK4; Euler: b_1 = 1; or the tableau)
    float cb[4] = {NST == 1 ? dt : dt / 6.0f, dt / 3.0f, dt / 3.0f, dt / 6.0f};
    float ca[4] = {0.5f * dt, 0.5f * dt, dt, 0.0f};
    if (TAB)
        for (int q = 0; q < 4; ++q) {
            cb[q] = v.rk_beta * v.rk_w[q] * dt;
            ca[q] = q < 3 ? v.rk_c[q] * dt : 0.0f;
        }
    float *seg0 = av.seg + av.seg_off[a.b];
    const long long seg_buf = (long long)min(ckpt, nsteps) * step_floats;  // floats of one segment buffer
    // per-segment FP32 and total FP64 weight gradients, column-slot order
    const long long cchunks = (long long)a.KC * nc;
    float4 *gpart = av.gpart + cslot0 / 4;
    double *gtot = av.gtot + cslot0;
    if (!fwd_cta) {
        for (long long c = tid; c < cchunks; c += nthr) gpart[c] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        for (long long c = tid; c < cchunks * 4; c += nthr) gtot[c] = 0.0;
    }
    // frames: global steps k in (step0, step0 + nsteps] with k % stride == 0
    const int stride = v.rec_stride;
    int frame = av.n_frames - 1;
    const float *dl = av.dLdV;
    if (!fwd_cta && stride > 0 && (step0 + nsteps) % stride == 0 && frame >= 0) {
        for (int i = tid; i < N; i += nthr) S.lam[i] += dl[(long long)frame * v.N + a.n0 + i];
        --frame;
    }
    __syncthreads();
    // segment c recomputed forward from its checkpoint into buffer c mod 2,
    // every step's four stages kept
    auto recompute = [&](int c) {
        const int k0 = c * ckpt, k1 = min(k0 + ckpt, nsteps);
        load_reduced(v, a, S, av.ck_full + (long long)c * av.dim,
                     av.ck_full_lo ? av.ck_full_lo + (long long)c * av.dim : nullptr, rp, gcode, nullptr);
        float *seg = seg0 + (long long)(c & 1) * seg_buf;
        for (int n = k0; n < k1; ++n) {
            fwd_step<true, NST, TAB>(v, a, S, stab, step0 + n, dt);
            float *dst = seg + (long long)(n - k0) * step_floats;
            if (NST == 4) {
                for (int q = tid; q < stage_floats / 4; q += nthr) ((float4 *)dst)[q] = stage_blk[q];
            } else {
                copy_stages<true>(S.sV, dst, N, M, NST);
            }
            __syncthreads();
        }
    };
    // segment c swept backward from buffer c mod 2
    auto sweep = [&](int c) {
        const int k0 = c * ckpt, k1 = min(k0 + ckpt, nsteps);
        const float *seg = seg0 + (long long)(c & 1) * seg_buf;
        for (int n = k1 - 1; n >= k0; --n) {
            const float *src = seg + (long long)(n - k0) * step_floats;
            if (NST == 4) {
                for (int q = tid; q < stage_floats / 4; q += nthr) stage_blk[q] = ((const float4 *)src)[q];
            } else {
                copy_stages<false>(S.sV, (float *)src, N, M, NST);
            }
            __syncthreads();
            rev_step<NST>(a, S, stab, cb, ca, gpart);
            if (stride > 0 && n > 0 && (step0 + n) % stride == 0 && frame >= 0) {
                for (int i = tid; i < N; i += nthr) S.lam[i] += dl[(long long)frame * v.N + a.n0 + i];
                --frame;
            }
            __syncthreads();
        }
        // fold the segment's partial sums into the FP64 totals
        for (long long q = tid; q < cchunks; q += nthr) {
            const float4 g = gpart[q];
            gtot[4 * q] += g.x;
            gtot[4 * q + 1] += g.y;
            gtot[4 * q + 2] += g.z;
            gtot[4 * q + 3] += g.w;
            gpart[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
        __syncthreads();
    };
    // pass 2: segments backward, rank 0 one segment ahead of rank 1; the
    // cluster barrier (release/acquire) hands each buffer over
    const int nseg = (nsteps + ckpt - 1) / ckpt;
    if (fwd_cta) recompute(nseg - 1);
    cluster_sync();
    for (int c = nseg - 1; c >= 0; --c) {
        if (fwd_cta) {
            if (c > 0) recompute(c - 1);
        } else {
            sweep(c);
        }
        cluster_sync();
    }
    if (fwd_cta) return;
    // outputs (rank 1): weight gradients in CSR order, neuron parameter partials
    {
        const int *ck = av.ck + cslot0;
        for (long long q = tid; q < cchunks * 4; q += nthr) {
            const int k = ck[q];
            if (k >= 0) av.grad_w[a.sbase + k] = (float)gtot[q];
        }
    }
    for (int i = tid; i < N; i += nthr) {
        for (int x = 0; x < 9; ++x) {
            const float2 c = S.gp[9 * i + x];
            av.gp_neuron[(long long)(a.n0 + i) * 9 + x] = (double)c.x + (double)c.y;
        }
        for (int x = 0; x < 4; ++x) av.grad_y0[(long long)x * v.N + a.n0 + i] = S.lam[x * N + i];
    }
}

// Sum of the per-neuron parameter gradients into the neuron-type table
// (fixed order: neuron index).
__global__ void adj_reduce_types(const int *neuron_type, long long N, const double *gp_neuron, int n_types,
                                 float *grad_np) {
    const int t = blockIdx.x, x = threadIdx.x;
    if (x >= 9) return;
    double acc = 0.0;
    for (long long i = 0; i < N; ++i)
        if (neuron_type[i] == t) acc += gp_neuron[i * 9 + x];
    grad_np[t * 9 + x] = (float)acc;
}

}  // namespace

long long adj_segment_floats(int method, int rk_ns, int N, int nt) {
    const int nst = method == PSST_METHOD_EULER ? 1 : method == PSST_METHOD_TABLEAU ? rk_ns : 4;
    return adj_step_floats(nst, N, (long long)N * nt);
}

long long adj_smem_need(int N, int nt, int n_items, int K, int n_citems, int KC) {
    return adj_smem_bytes(N, N * nt, n_items, K, n_citems, KC);
}

cudaError_t adj_launch(const NetView &v, const AdjView &av, long long step0, int nsteps, int smem, int n_types,
                       float *grad_np, cudaStream_t stream) {
    // RK4 (four stages a step), forward Euler (one) or a tableau of 1..4 stages
    void (*kern)(NetView, AdjView, long long, int) = v.method == PSST_METHOD_EULER ? adj_kernel<1, false>
                                                                                    : adj_kernel<4, false>;
    if (v.method == PSST_METHOD_TABLEAU)
        kern = v.rk_ns == 1   ? adj_kernel<1, true>
               : v.rk_ns == 2 ? adj_kernel<2, true>
               : v.rk_ns == 3 ? adj_kernel<3, true>
                              : adj_kernel<4, true>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    // one cluster of two CTAs per network: forward recompute and reverse sweep
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(2 * v.n_nets);
    cfg.blockDim = dim3(ADJ_THREADS);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, v, av, step0, nsteps);
    if (e != cudaSuccess) return e;
    adj_reduce_types<<<n_types, 32, 0, stream>>>(v.neuron_type, v.N, av.gp_neuron, n_types, grad_np);
    return cudaGetLastError();
}

}  // namespace psst
