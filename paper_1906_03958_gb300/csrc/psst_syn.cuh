// Synapses of a block of CSR rows held in shared memory in a padded,
// 4-wide chunk layout, and the S-phase (synaptic current of every owned
// row at one RK4 stage) over that layout.  Shared by the CTA/cluster kernel
// and the grid-wide kernel.
//
// Layout.  Each row's synapses are split into its first-order gates and its
// second-order (r, s) pairs; each part is padded to a multiple of 4 with
// inert entries (w = 0, gate 0, coefficient index 0).  Chunk c holds 4
// synapses as float4 r, float4 w, float4 wE (= w * E of its type),
// ushort4 id (coefficient index pre * n_types + type) and, second order only,
// float4 s.  Row i owns chunks [cb[i], cm[i]) (first order) and
// [cm[i], cb[i+1]) (second order).
//
// Current.  I_syn,i = sum_k w_k G_k (V_i - E_k) = V_i A_i - B_i with
// A_i = sum_k w_k G_k and B_i = sum_k (w_k E_k) G_k, accumulated per lane and
// summed over the row's G lanes by a shuffle tree (fixed order).
#pragma once

#include "psst_device.cuh"

namespace psst {

struct RowChunks {
    int nrows;
    int *cb;       // [nrows+1]
    int *cm;       // [nrows]
    float4 *r, *s, *w, *we;
    ushort4 *id;
};

// Shared-memory bytes of the synapse part for `chunks` chunks and `nrows` rows.
__host__ __device__ inline long long syn_smem_bytes(long long chunks, int nrows, bool has2) {
    const long long per = has2 ? 16 * 4 + 8 : 16 * 3 + 8;
    return chunks * per + 8LL * nrows + 32;
}

// Number of chunks a row needs (first + second order parts padded to 4).
__host__ __device__ inline int row_chunks(int n1, int n2) { return (n1 + 3) / 4 + (n2 + 3) / 4; }

// Carve the chunk arrays out of `base` (16-aligned) for `chunks` chunks.
__device__ inline RowChunks carve_rows(unsigned char *base, int nrows, int chunks, bool has2) {
    RowChunks rc;
    rc.nrows = nrows;
    unsigned char *p = base;
    rc.r = (float4 *)p;
    p += 16LL * chunks;
    rc.w = (float4 *)p;
    p += 16LL * chunks;
    rc.we = (float4 *)p;
    p += 16LL * chunks;
    rc.s = has2 ? (float4 *)p : nullptr;
    if (has2) p += 16LL * chunks;
    rc.id = (ushort4 *)p;
    p += 8LL * chunks;
    rc.cb = (int *)p;
    p += 4LL * (nrows + 1);
    rc.cm = (int *)p;
    return rc;
}

// Block-wide exclusive prefix sum of cnt[0..n) into out[0..n] (out[n] = total),
// executed by warp 0 in 32-wide strips; all threads must call it.
__device__ inline void block_scan(const int *cnt, int *out, int n) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int carry = 0;
        for (int base = 0; base < n; base += 32) {
            const int i = base + lane;
            const int v = i < n ? cnt[i] : 0;
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (i < n) out[i] = carry + x - v;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) out[n] = carry;
    }
    __syncthreads();
}

// Fill the chunk layout for rows [row0, row0 + nrows) of a network from the
// global CSR arrays (synapse k of the network at offset k - sbase).  `tmp`
// is scratch shared memory of nrows + 1 ints.  `stab` is the synapse-type
// table (kind at SP_KIND, E at SP_E).
template <bool HAS2>
__device__ void load_rows(RowChunks &rc, const NetView &v, long long row_g0, long long sbase, int row0,
                          const float *gr, const float *gs, const float *gw, const uint32_t *gcode,
                          const float *stab, int *tmp) {
    const int tid = threadIdx.x, nthr = blockDim.x, nrows = rc.nrows;
    // per-row counts of first/second-order synapses
    for (int i = tid; i < nrows; i += nthr) {
        const long long k0 = v.row_ptr[row_g0 + row0 + i] - sbase, k1 = v.row_ptr[row_g0 + row0 + i + 1] - sbase;
        int n2 = 0;
        if (HAS2)
            for (long long k = k0; k < k1; ++k) n2 += stab[(gcode[k] >> 24) * 9 + SP_KIND] != 0.0f;
        const int n1 = (int)(k1 - k0) - n2;
        tmp[i] = row_chunks(n1, n2);
        rc.cm[i] = (n1 + 3) / 4;  // first-order chunk count, offset fixed below
    }
    __syncthreads();
    block_scan(tmp, rc.cb, nrows);
    const int chunks = rc.cb[nrows];
    for (int c = tid; c < chunks; c += nthr) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        rc.r[c] = z;
        rc.w[c] = z;
        rc.we[c] = z;
        if (HAS2) rc.s[c] = z;
        rc.id[c] = make_ushort4(0, 0, 0, 0);
    }
    for (int i = tid; i < nrows; i += nthr) rc.cm[i] += rc.cb[i];
    __syncthreads();
    for (int i = tid; i < nrows; i += nthr) {
        const long long k0 = v.row_ptr[row_g0 + row0 + i] - sbase, k1 = v.row_ptr[row_g0 + row0 + i + 1] - sbase;
        int p1 = rc.cb[i] * 4, p2 = rc.cm[i] * 4;
        float *R = (float *)rc.r, *W = (float *)rc.w, *WE = (float *)rc.we, *Sg = (float *)rc.s;
        unsigned short *ID = (unsigned short *)rc.id;
        for (long long k = k0; k < k1; ++k) {
            const uint32_t code = gcode[k];
            const int tau = (int)(code >> 24);
            const bool second = HAS2 && stab[tau * 9 + SP_KIND] != 0.0f;
            const int p = second ? p2++ : p1++;
            const float w = gw[k];
            R[p] = gr[k];
            W[p] = w;
            WE[p] = w * stab[tau * 9 + SP_E];
            ID[p] = (unsigned short)(code & 0xFFFFFFu);
            if (HAS2) Sg[p] = second ? gs[k] : 0.0f;
        }
    }
    __syncthreads();
}

// Write the owned synapses back to the global CSR arrays, applying the last
// step's gate map (fin1: r-map, fin2: s-map), in the same slot order as
// load_rows.  fin tables are indexed by the coefficient index.
template <bool HAS2, class Fin>
__device__ void store_rows(const RowChunks &rc, const NetView &v, long long row_g0, long long sbase, int row0,
                           float *gr, float *gs, const uint32_t *gcode, const float *stab, const Fin &fin) {
    const int tid = threadIdx.x, nthr = blockDim.x, nrows = rc.nrows;
    for (int i = tid; i < nrows; i += nthr) {
        const long long k0 = v.row_ptr[row_g0 + row0 + i] - sbase, k1 = v.row_ptr[row_g0 + row0 + i + 1] - sbase;
        int p1 = rc.cb[i] * 4, p2 = rc.cm[i] * 4;
        const float *R = (const float *)rc.r, *Sg = (const float *)rc.s;
        for (long long k = k0; k < k1; ++k) {
            const uint32_t code = gcode[k];
            const int tau = (int)(code >> 24);
            const int ci = (int)(code & 0xFFFFFFu);
            const bool second = HAS2 && stab[tau * 9 + SP_KIND] != 0.0f;
            const int p = second ? p2++ : p1++;
            const float r0 = R[p];
            const float2 F = fin.r(ci);
            gr[k] = fmaf(F.y, r0, F.x);
            if (HAS2 && second) {
                const float4 F2 = fin.s(ci);
                gs[k] = fmaf(F2.z, Sg[p], fmaf(F2.y, r0, F2.x));
            }
        }
    }
}

// One synapse of the current stage: gate value from the affine map, then
// accumulate A += w G, B += wE G.  ST == 0 applies the previous step's final
// map and stores the new step-start gate.
template <bool FIRST_STAGE>
__device__ __forceinline__ void syn1(float &r, float w, float we, float2 F, float &A, float &B) {
    const float g = fmaf(F.y, r, F.x);
    if (FIRST_STAGE) r = g;
    A = fmaf(w, g, A);
    B = fmaf(we, g, B);
}

template <bool FIRST_STAGE>
__device__ __forceinline__ void syn2(float &r, float &s, float w, float we, float2 F, float4 F2, float &A,
                                     float &B) {
    const float rr = fmaf(F.y, r, F.x);
    const float ss = fmaf(F2.z, s, fmaf(F2.y, r, F2.x));
    if (FIRST_STAGE) {
        r = rr;
        s = ss;
    }
    const float s2 = ss * ss, s4 = s2 * s2;
    const float g = __fdividef(s4, s4 + F2.w);
    A = fmaf(w, g, A);
    B = fmaf(we, g, B);
}

// S-phase over the owned rows: lanes of a G-lane group stride the row's
// chunks; row sums go to out(row, value).  Coef supplies r(ci) (float2
// affine r-map of this stage) and s(ci) (float4 s-map, w = Kd).
template <int ST, bool HAS2, class Coef, class Out>
__device__ __forceinline__ void sphase(const RowChunks &rc, const float *Vrow, const Coef &cf, int G,
                                       const Out &out) {
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int ngroups = nthr / G, gid = tid / G, gl = tid % G;
    const int nrows = rc.nrows;
    for (int base = 0; base < nrows; base += ngroups) {
        const int row = base + gid;
        float A = 0.0f, B = 0.0f;
        if (row < nrows) {
            const int c0 = rc.cb[row], cmid = rc.cm[row];
            for (int c = c0 + gl; c < cmid; c += G) {
                float4 r = rc.r[c];
                const float4 w = rc.w[c], we = rc.we[c];
                const ushort4 id = rc.id[c];
                syn1<ST == 0>(r.x, w.x, we.x, cf.r(id.x), A, B);
                syn1<ST == 0>(r.y, w.y, we.y, cf.r(id.y), A, B);
                syn1<ST == 0>(r.z, w.z, we.z, cf.r(id.z), A, B);
                syn1<ST == 0>(r.w, w.w, we.w, cf.r(id.w), A, B);
                if (ST == 0) rc.r[c] = r;
            }
            if (HAS2) {
                const int c1 = rc.cb[row + 1];
                for (int c = cmid + gl; c < c1; c += G) {
                    float4 r = rc.r[c], s = rc.s[c];
                    const float4 w = rc.w[c], we = rc.we[c];
                    const ushort4 id = rc.id[c];
                    syn2<ST == 0>(r.x, s.x, w.x, we.x, cf.r(id.x), cf.s(id.x), A, B);
                    syn2<ST == 0>(r.y, s.y, w.y, we.y, cf.r(id.y), cf.s(id.y), A, B);
                    syn2<ST == 0>(r.z, s.z, w.z, we.z, cf.r(id.z), cf.s(id.z), A, B);
                    syn2<ST == 0>(r.w, s.w, w.w, we.w, cf.r(id.w), cf.s(id.w), A, B);
                    if (ST == 0) {
                        rc.r[c] = r;
                        rc.s[c] = s;
                    }
                }
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1)
            if (off < G) {
                A += __shfl_xor_sync(0xffffffffu, A, off);
                B += __shfl_xor_sync(0xffffffffu, B, off);
            }
        if (row < nrows && gl == 0) out(row, fmaf(Vrow[row], A, -B));
    }
}

// Gate-map update of one (presynaptic neuron j, synapse type tau) pair at
// stage ST from the stage-ST potential V of j.  cur/acc hold this stage's
// map and the running RK4 sum; writes the next stage's map into cur (ST < 3)
// or the step's final map into fin (ST == 3).  The s-map's fourth component
// carries Kd (1 for first-order types, whose s-map is never used).
template <int ST, bool HAS2>
__device__ __forceinline__ void coef_update(const float *sp, float V, float dt, float2 &cur, float2 &acc,
                                            float2 &fin, float4 &cur2, float4 &acc2, float4 &fin2) {
    constexpr float WGT = (ST == 0 || ST == 3) ? 1.0f : 2.0f;
    const float cnext = (ST == 2) ? dt : 0.5f * dt;
    const float dt6 = dt * (1.0f / 6.0f);
    const float T = transmitter(V, sp[SP_VP], sp[SP_KP]);  // table holds 1/Kp
    const float a_ = sp[SP_A] * T, bb = a_ + sp[SP_B];
    float P = 0.0f, Q = 1.0f, U = 0.0f, X = 0.0f, Z = 1.0f;
    if (ST > 0) {
        P = cur.x;
        Q = cur.y;
        if (HAS2) {
            U = cur2.x;
            X = cur2.y;
            Z = cur2.z;
        }
    }
    const float kP = fmaf(-bb, P, a_), kQ = -bb * Q;
    float2 A1 = make_float2(kP, kQ);
    if (ST > 0) A1 = make_float2(fmaf(WGT, kP, acc.x), fmaf(WGT, kQ, acc.y));
    if (ST < 3) {
        acc = A1;
        cur = make_float2(cnext * kP, fmaf(cnext, kQ, 1.0f));
    } else {
        fin = make_float2(dt6 * A1.x, fmaf(dt6, A1.y, 1.0f));
    }
    if (HAS2) {
        const float K3 = sp[SP_K3], K4 = sp[SP_K4];
        const float Kd = sp[SP_KIND] != 0.0f ? sp[SP_KD] : 1.0f;
        const float kU = fmaf(K3, P, -K4 * U), kX = fmaf(K3, Q, -K4 * X), kZ = -K4 * Z;
        float4 A2 = make_float4(kU, kX, kZ, 0.0f);
        if (ST > 0) A2 = make_float4(fmaf(WGT, kU, acc2.x), fmaf(WGT, kX, acc2.y), fmaf(WGT, kZ, acc2.z), 0.0f);
        if (ST < 3) {
            acc2 = A2;
            cur2 = make_float4(cnext * kU, cnext * kX, fmaf(cnext, kZ, 1.0f), Kd);
        } else {
            fin2 = make_float4(dt6 * A2.x, dt6 * A2.y, fmaf(dt6, A2.z, 1.0f), Kd);
        }
    }
}

// Right-hand side and stage update of neuron i at stage ST.  y0/acc/ys hold
// [4][N] (ys rows 1..3 = stage m, h, n); V is the stage potential; returns
// the potential of the next stage (ST < 3) or of the new step start.
template <int ST>
__device__ __forceinline__ float neuron_update(int i, int N, float V, float *y0, float *acc, float *ys,
                                               const float *prm, float iext, float isyn, float dt) {
    constexpr float WGT = (ST == 0 || ST == 3) ? 1.0f : 2.0f;
    const float cnext = (ST == 2) ? dt : 0.5f * dt;
    const float dt6 = dt * (1.0f / 6.0f);
    const float m = ys[N + i], h = ys[2 * N + i], n = ys[3 * N + i];
    const Rates q = hh_rates(V);
    const float m3h = m * m * m * h, n2 = n * n, n4 = n2 * n2;
    const float iion = prm[NP_GNA * N + i] * m3h * (V - prm[NP_ENA * N + i]) +
                       prm[NP_GK * N + i] * n4 * (V - prm[NP_EK * N + i]) +
                       prm[NP_GL * N + i] * (V - prm[NP_EL * N + i]) +
                       prm[NP_GKL * N + i] * (V - prm[NP_EKL * N + i]);
    float d[4];
    d[0] = (iext - iion - isyn) * prm[NP_C * N + i];  // prm row 0 holds 1/C
    d[1] = q.am * (1.0f - m) - q.bm * m;
    d[2] = q.ah * (1.0f - h) - q.bh * h;
    d[3] = q.an * (1.0f - n) - q.bn * n;
    float vnext = 0.0f;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
        const int ix = x * N + i;
        const float ac = (ST == 0) ? d[x] : fmaf(WGT, d[x], acc[ix]);
        float yn;
        if (ST < 3) {
            acc[ix] = ac;
            yn = fmaf(cnext, d[x], y0[ix]);
        } else {
            yn = fmaf(dt6, ac, y0[ix]);
            y0[ix] = yn;
        }
        if (x == 0) vnext = yn;
        else ys[ix] = yn;
    }
    return vnext;
}

}  // namespace psst
