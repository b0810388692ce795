// CTA-resident RK4 integration: one thread block owns one network at a time
// and keeps it on chip (shared memory) for all of the launch's steps, then
// takes the next network from a device work queue.  One launch integrates a
// whole ragged batch (thousands of networks of uneven size).
//
// Per RK4 step (classic tableau, Sec. "Brain simulations as computational
// graphs", RK4 paragraph) and per stage s = 0..3:
//   S-phase  (row groups of G lanes, one CSR row = one postsynaptic neuron):
//            I_syn,i = sum_k w_k G(r_k^(s)) (V_i^(s) - E_k), warp-shuffle sum;
//   N-phase  (one thread per neuron): HH right-hand side, RK4 stage/combine
//            for V, m, h, n, and the per-presynaptic-neuron coefficients of
//            the synaptic gates for the next stage.
//
// Synaptic gates.  A gate's equation dr/dt = a T_j (1 - r) - b r is affine in
// r with coefficients set by its presynaptic neuron j alone, so every RK4
// stage value of every gate from j is an affine function of the gate's
// step-start value:  r^(s) = P_s[j] + Q_s[j] r0  (and for second-order
// pairs s^(s) = U_s[j] + X_s[j] r0 + Z_s[j] s0).  The coefficients are
// propagated once per presynaptic neuron and stage (O(N) work) and each
// synapse evaluates its stage value with one FMA; the step-end map
// r <- P + Q r0 is applied lazily at the next step's first stage.  This is
// the same RK4 map as the textbook stage recursion, evaluated in a
// different (algebraically identical) order.
#include <cuda_runtime.h>

#include "psst_device.cuh"
#include "psst_internal.h"

namespace psst {

namespace {

struct Ctx {
    int N, S, nt, G, n0, b;
    float dt;
    float2 *c1cur, *c1fin, *c1acc;
    float4 *c2cur, *c2fin, *c2acc;
    float *y0, *ys, *acc, *prm, *iext, *isyn;
    int *rowp;
    float *r, *s, *w;
    const uint32_t *code;
};

// Stage s of one RK4 step: S-phase, barrier, N-phase, barrier.
template <int ST, bool HAS2>
__device__ __forceinline__ void rk4_stage(const NetView &v, const Ctx &c, const float *stab,
                                          long long step) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int G = c.G, ngroups = nthr / G, gid = tid / G, gl = tid % G;
    const int N = c.N, nt = c.nt;

    // ---- S-phase: synaptic current onto every row at stage ST
    for (int base = 0; base < N; base += ngroups) {
        const int row = base + gid;
        float a = 0.0f;
        if (row < N) {
            const float Vi = c.ys[row];
            const int k1 = c.rowp[row + 1];
            for (int k = c.rowp[row] + gl; k < k1; k += G) {
                const uint32_t code = c.code[k];
                const int ci = (int)(code & 0xFFFFFFu);
                const int tau = (int)(code >> 24);
                const float r0 = c.r[k];
                float rr, ss = 0.0f;
                if (ST == 0) {
                    const float2 F = c.c1fin[ci];
                    rr = fmaf(F.y, r0, F.x);
                    c.r[k] = rr;
                    if (HAS2) {
                        const float4 F2 = c.c2fin[ci];
                        ss = fmaf(F2.z, c.s[k], fmaf(F2.y, r0, F2.x));
                        c.s[k] = ss;
                    }
                } else {
                    const float2 P = c.c1cur[ci];
                    rr = fmaf(P.y, r0, P.x);
                    if (HAS2) {
                        const float4 U = c.c2cur[ci];
                        ss = fmaf(U.z, c.s[k], fmaf(U.y, r0, U.x));
                    }
                }
                float g = rr;
                if (HAS2) {
                    if (stab[tau * 9 + SP_KIND] != 0.0f) {
                        const float s2 = ss * ss, s4 = s2 * s2;
                        g = __fdividef(s4, s4 + stab[tau * 9 + SP_KD]);
                    }
                }
                a = fmaf(c.w[k] * g, Vi - stab[tau * 9 + SP_E], a);
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            if (off < G) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (row < N && gl == 0) c.isyn[row] = a;
    }
    __syncthreads();

    // ---- N-phase: neuron right-hand side and stage update
    constexpr float WGT = (ST == 0 || ST == 3) ? 1.0f : 2.0f;
    const float cnext = (ST == 2) ? c.dt : 0.5f * c.dt;
    const float dt6 = c.dt * (1.0f / 6.0f);
    for (int i = tid; i < N; i += nthr) {
        const float V = c.ys[i], m = c.ys[N + i], h = c.ys[2 * N + i], n = c.ys[3 * N + i];
        const float *p = c.prm;
        const Rates q = hh_rates(V);
        const float m3h = m * m * m * h, n2 = n * n, n4 = n2 * n2;
        const float iion = p[NP_GNA * N + i] * m3h * (V - p[NP_ENA * N + i]) +
                           p[NP_GK * N + i] * n4 * (V - p[NP_EK * N + i]) +
                           p[NP_GL * N + i] * (V - p[NP_EL * N + i]) +
                           p[NP_GKL * N + i] * (V - p[NP_EKL * N + i]);
        float d[4];
        d[0] = (c.iext[i] - iion - c.isyn[i]) * p[NP_C * N + i];  // prm[0] holds 1/C
        d[1] = q.am * (1.0f - m) - q.bm * m;
        d[2] = q.ah * (1.0f - h) - q.bh * h;
        d[3] = q.an * (1.0f - n) - q.bn * n;
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const int ix = x * N + i;
            const float ac = (ST == 0) ? d[x] : fmaf(WGT, d[x], c.acc[ix]);
            if (ST < 3) {
                c.acc[ix] = ac;
                c.ys[ix] = fmaf(cnext, d[x], c.y0[ix]);
            } else {
                const float yn = fmaf(dt6, ac, c.y0[ix]);
                c.y0[ix] = yn;
                c.ys[ix] = yn;
            }
        }
        if (ST == 3 && v.rec_stride > 0 && ((step + 1) % v.rec_stride) == 0) {
            const long long frame = (step + 1) / v.rec_stride - 1;
            v.rec[(frame % v.rec_cap) * v.N + c.n0 + i] = c.y0[i];
        }
        // gate coefficients of synapses whose presynaptic neuron is i
        for (int tau = 0; tau < nt; ++tau) {
            const float *sp = stab + tau * 9;
            const float T = transmitter(V, sp[SP_VP], sp[SP_KP]);  // table holds 1/Kp
            const float a_ = sp[SP_A] * T, bb = a_ + sp[SP_B];
            const int ci = i * nt + tau;
            float P = 0.0f, Q = 1.0f, U = 0.0f, X = 0.0f, Z = 1.0f;
            if (ST > 0) {
                const float2 pq = c.c1cur[ci];
                P = pq.x;
                Q = pq.y;
                if (HAS2) {
                    const float4 u = c.c2cur[ci];
                    U = u.x;
                    X = u.y;
                    Z = u.z;
                }
            }
            const float kP = fmaf(-bb, P, a_), kQ = -bb * Q;
            float2 A1 = make_float2(kP, kQ);
            if (ST > 0) {
                const float2 o = c.c1acc[ci];
                A1 = make_float2(fmaf(WGT, kP, o.x), fmaf(WGT, kQ, o.y));
            }
            if (ST < 3) {
                c.c1acc[ci] = A1;
                c.c1cur[ci] = make_float2(cnext * kP, fmaf(cnext, kQ, 1.0f));
            } else {
                c.c1fin[ci] = make_float2(dt6 * A1.x, fmaf(dt6, A1.y, 1.0f));
            }
            if (HAS2) {
                const float K3 = sp[SP_K3], K4 = sp[SP_K4];
                const float kU = fmaf(K3, P, -K4 * U), kX = fmaf(K3, Q, -K4 * X), kZ = -K4 * Z;
                float4 A2 = make_float4(kU, kX, kZ, 0.0f);
                if (ST > 0) {
                    const float4 o = c.c2acc[ci];
                    A2 = make_float4(fmaf(WGT, kU, o.x), fmaf(WGT, kX, o.y), fmaf(WGT, kZ, o.z), 0.0f);
                }
                if (ST < 3) {
                    c.c2acc[ci] = A2;
                    c.c2cur[ci] = make_float4(cnext * kU, cnext * kX, fmaf(cnext, kZ, 1.0f), 0.0f);
                } else {
                    c.c2fin[ci] = make_float4(dt6 * A2.x, dt6 * A2.y, fmaf(dt6, A2.z, 1.0f), 0.0f);
                }
            }
        }
    }
    __syncthreads();
}

template <bool SMEM, bool HAS2>
__device__ void integrate_net(const NetView &v, int b, long long step0, int nsteps, int G,
                              unsigned char *smem, const float *stab) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    Ctx c;
    c.b = b;
    c.n0 = v.net_off[b];
    c.N = v.net_off[b + 1] - c.n0;
    const long long sbase = v.row_ptr[c.n0];
    c.S = (int)(v.row_ptr[c.n0 + c.N] - sbase);
    c.nt = v.n_stypes;
    c.G = G;
    c.dt = v.dt;
    const int N = c.N, S = c.S, M = N * c.nt;
    const Layout L = make_layout(N, S, c.nt, HAS2, SMEM);
    c.c1cur = (float2 *)(smem + L.c1cur);
    c.c1fin = (float2 *)(smem + L.c1fin);
    c.c1acc = (float2 *)(smem + L.c1acc);
    c.c2cur = HAS2 ? (float4 *)(smem + L.c2cur) : nullptr;
    c.c2fin = HAS2 ? (float4 *)(smem + L.c2fin) : nullptr;
    c.c2acc = HAS2 ? (float4 *)(smem + L.c2acc) : nullptr;
    c.y0 = (float *)(smem + L.y0);
    c.ys = (float *)(smem + L.ys);
    c.acc = (float *)(smem + L.acc);
    c.prm = (float *)(smem + L.prm);
    c.iext = (float *)(smem + L.iext);
    c.isyn = (float *)(smem + L.isyn);
    c.rowp = (int *)(smem + L.rowp);

    float *gV = v.state + c.n0;
    float *gr = v.state + 4 * v.N + sbase;
    float *gs = v.state + 4 * v.N + v.S + sbase;
    const float *gw = v.weight + sbase;
    const uint32_t *gcode = v.syn_code + sbase;

    for (int i = tid; i < N; i += nthr) {
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const float y = gV[(long long)x * v.N + i];
            c.y0[x * N + i] = y;
            c.ys[x * N + i] = y;
        }
        const float *p = v.nparams + (long long)v.neuron_type[c.n0 + i] * PSST_NEURON_NPARAM;
        c.prm[NP_C * N + i] = 1.0f / p[NP_C];
#pragma unroll
        for (int x = 1; x < PSST_NEURON_NPARAM; ++x) c.prm[x * N + i] = p[x];
        c.rowp[i] = (int)(v.row_ptr[c.n0 + i] - sbase);
    }
    if (tid == 0) c.rowp[N] = S;
    for (int k = tid; k < M; k += nthr) {
        c.c1fin[k] = make_float2(0.0f, 1.0f);
        if (HAS2) c.c2fin[k] = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
    }
    if (SMEM) {
        c.r = (float *)(smem + L.r);
        c.w = (float *)(smem + L.w);
        uint32_t *cd = (uint32_t *)(smem + L.code);
        c.s = HAS2 ? (float *)(smem + L.s) : nullptr;
        for (int k = tid; k < S; k += nthr) {
            c.r[k] = gr[k];
            c.w[k] = gw[k];
            cd[k] = gcode[k];
            if (HAS2) c.s[k] = gs[k];
        }
        c.code = cd;
    } else {
        c.r = gr;
        c.s = gs;
        c.w = const_cast<float *>(gw);
        c.code = gcode;
    }
    __syncthreads();

    for (int it = 0; it < nsteps; ++it) {
        const long long step = step0 + it;
        for (int i = tid; i < N; i += nthr) c.iext[i] = input_current(v, b, (long long)c.n0 + i, step);
        // iext is consumed in the N-phase, after the S-phase barrier
        rk4_stage<0, HAS2>(v, c, stab, step);
        rk4_stage<1, HAS2>(v, c, stab, step);
        rk4_stage<2, HAS2>(v, c, stab, step);
        rk4_stage<3, HAS2>(v, c, stab, step);
    }

    // write back: apply the last step's gate map, store neuron state
    for (int k = tid; k < S; k += nthr) {
        const uint32_t code = c.code[k];
        const int ci = (int)(code & 0xFFFFFFu);
        const float r0 = c.r[k];
        const float2 F = c.c1fin[ci];
        gr[k] = fmaf(F.y, r0, F.x);
        if (HAS2) {
            const float4 F2 = c.c2fin[ci];
            gs[k] = fmaf(F2.z, c.s[k], fmaf(F2.y, r0, F2.x));
        }
    }
    bool bad = false;
    for (int i = tid; i < N; i += nthr) {
#pragma unroll
        for (int x = 0; x < 4; ++x) {
            const float y = c.y0[x * N + i];
            bad |= !isfinite(y);
            gV[(long long)x * v.N + i] = y;
        }
    }
    if (bad) set_error(v.err, PSST_ERR_NONFINITE);
}

__global__ void __launch_bounds__(1024) cta_kernel(NetView v, long long step0, int nsteps, int G) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float stab[PSST_MAX_SYN_TYPES * PSST_SYN_NPARAM];
    __shared__ int s_next;
    for (int i = threadIdx.x; i < v.n_stypes * PSST_SYN_NPARAM; i += blockDim.x) {
        float x = v.sparams[i];
        if (i % PSST_SYN_NPARAM == SP_KP) x = 1.0f / x;  // stored as 1/Kp
        stab[i] = x;
    }
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_next = atomicAdd(v.work_counter, 1);
        __syncthreads();
        const int w = s_next;
        if (w >= v.n_nets) return;
        const int b = v.order[w];
        const uint8_t fl = v.net_flags[b];
        if (fl & NET_FITS_SMEM) {
            if (fl & NET_HAS2) integrate_net<true, true>(v, b, step0, nsteps, G, smem, stab);
            else integrate_net<true, false>(v, b, step0, nsteps, G, smem, stab);
        } else {
            if (fl & NET_HAS2) integrate_net<false, true>(v, b, step0, nsteps, G, smem, stab);
            else integrate_net<false, false>(v, b, step0, nsteps, G, smem, stab);
        }
    }
}

}  // namespace

int cta_max_smem(int device) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess)
        return -1;
    // the kernel's static shared memory
    return v - (int)(PSST_MAX_SYN_TYPES * PSST_SYN_NPARAM * sizeof(float) + 16);
}

cudaError_t cta_occupancy(int block, int smem, int *blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, cta_kernel, block, smem);
}

cudaError_t cta_launch(const NetView &v, long long step0, int nsteps, int grid, int block, int G,
                       int smem, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(v.work_counter, 0, sizeof(int), stream);
    if (e != cudaSuccess) return e;
    cta_kernel<<<grid, block, smem, stream>>>(v, step0, nsteps, G);
    return cudaGetLastError();
}

}  // namespace psst
