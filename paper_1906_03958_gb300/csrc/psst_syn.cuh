// Synapses of a block of CSR rows held in shared memory as fixed-size work
// items, the S-phase over them, and the per-neuron / per-gate-map stage
// updates.  Shared by the CTA/cluster kernel and the grid-wide kernel.
//
// Work items.  Each row's synapses are split into its first-order gates and
// its second-order (r, s) pairs.  Each part is cut into items of K chunks of
// 4 synapses (the last item of a row padded with inert entries: w = 0,
// gate 0, coefficient index 0).  All rows' first-order items form list 1,
// all second-order items list 2.  A list of n items is stored slot-major:
// chunk j of item t sits at j * n + t, so the lanes of a warp read
// consecutive 16-byte slots.  Per chunk: float4 r, w, wE (= w * E of its
// type), ushort4 coefficient index (pre * n_types + type), and float4 s for
// list 2.  Row i owns items [ib1[i], ib1[i+1]) of list 1 and
// [ib2[i], ib2[i+1]) of list 2.
//
// S-phase.  One thread per item accumulates A = sum w G and B = sum wE G
// over its K chunks and stores them; after a barrier the thread of neuron i
// adds its row's item partials in item order and forms
// I_syn,i = V_i A_i - B_i.  The summation order is fixed by the layout, so
// results are bitwise reproducible.
#pragma once

#include "psst_device.cuh"

namespace psst {

struct Items {
    int nrows, K, n1, n2;
    int *ib1, *ib2;           // [nrows+1] item offsets of each row in list 1 / list 2
    float4 *r, *s, *w, *we;   // [K * (n1 + n2)] chunks, list 1 then list 2 (s: list 2 only)
    ushort4 *id;
    float *pa, *pb;           // [n1 + n2] item partial sums
};

// Items of a row part with n synapses.
__host__ __device__ inline int part_items(int n, int K) { return (n + 4 * K - 1) / (4 * K); }

// Shared-memory bytes of the items of one block of rows.
__host__ __device__ inline long long items_smem_bytes(int n1, int n2, int K, int nrows, bool has2) {
    const long long c1 = (long long)K * n1, c2 = (long long)K * n2;
    long long b = (c1 + c2) * (16 * 3 + 8) + (has2 ? 16 * c2 : 0);
    b += 8LL * (n1 + n2);          // partials
    b += 8LL * (nrows + 1) + 64;   // row item offsets + alignment slack
    return b;
}

__device__ inline Items carve_items(unsigned char *base, int nrows, int K, int n1, int n2, bool has2) {
    Items it;
    it.nrows = nrows;
    it.K = K;
    it.n1 = n1;
    it.n2 = n2;
    const long long c = (long long)K * (n1 + n2);
    unsigned char *p = base;
    it.r = (float4 *)p;
    p += 16 * c;
    it.w = (float4 *)p;
    p += 16 * c;
    it.we = (float4 *)p;
    p += 16 * c;
    it.s = has2 ? (float4 *)p - (long long)K * n1 : nullptr;  // indexed like the others; list 2 only
    if (has2) p += 16LL * K * n2;
    it.id = (ushort4 *)p;
    p += 8 * c;
    it.pa = (float *)p;
    p += 4LL * (n1 + n2);
    it.pb = (float *)p;
    p += 4LL * (n1 + n2);
    it.ib1 = (int *)p;
    p += 4LL * (nrows + 1);
    it.ib2 = (int *)p;
    return it;
}

// Block-wide exclusive prefix sum of cnt[0..n) into out[0..n] (out[n] = total),
// executed by warp 0 in 32-wide strips; all threads must call it.
__device__ inline void block_scan(const int *cnt, int *out, int n) {
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        int carry = 0;
        for (int base = 0; base < n; base += 32) {
            const int i = base + lane;
            const int x0 = i < n ? cnt[i] : 0;
            int x = x0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            if (i < n) out[i] = carry + x - x0;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
        if (lane == 0) out[n] = carry;
    }
    __syncthreads();
}

// Slot of the m-th synapse of a row part that starts at item `ib` of a list
// with n items (chunk index * 4 + lane within the chunk).
__device__ __forceinline__ long long item_slot(int ib, int m, int K, int n, int base_chunk) {
    const int t = ib + m / (4 * K);
    const int j = (m % (4 * K)) >> 2;
    return ((long long)base_chunk + (long long)j * n + t) * 4 + (m & 3);
}

__device__ __forceinline__ bool second_order(const float *stab, uint32_t code) {
    return stab[(code >> 24) * 9 + SP_KIND] != 0.0f;
}

// Fill the items of rows [row0, row0 + nrows) of a network from the global
// CSR arrays (synapse k of the network at offset k - sbase; rows of the
// network start at global row row_g0).  tmp: shared scratch of 2 (nrows + 1)
// ints.  stab: synapse-type table.
template <bool HAS2>
__device__ void load_items(Items &it, const NetView &v, long long row_g0, long long sbase, int row0,
                           const float *gr, const float *gs, const float *gw, const uint32_t *gcode,
                           const float *stab, int *tmp) {
    const int tid = threadIdx.x, nthr = blockDim.x, nrows = it.nrows, K = it.K;
    int *c1 = tmp, *c2 = tmp + nrows + 1;
    for (int i = tid; i < nrows; i += nthr) {
        const long long k0 = v.row_ptr[row_g0 + row0 + i] - sbase, k1 = v.row_ptr[row_g0 + row0 + i + 1] - sbase;
        int n2 = 0;
        if (HAS2)
            for (long long k = k0; k < k1; ++k) n2 += second_order(stab, gcode[k]);
        c1[i] = part_items((int)(k1 - k0) - n2, K);
        c2[i] = part_items(n2, K);
    }
    __syncthreads();
    block_scan(c1, it.ib1, nrows);
    block_scan(c2, it.ib2, nrows);
    const long long chunks = (long long)K * (it.n1 + it.n2);
    for (long long c = tid; c < chunks; c += nthr) {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        it.r[c] = z;
        it.w[c] = z;
        it.we[c] = z;
        if (HAS2 && c >= (long long)K * it.n1) it.s[c] = z;
        it.id[c] = make_ushort4(0, 0, 0, 0);
    }
    __syncthreads();
    float *R = (float *)it.r, *W = (float *)it.w, *WE = (float *)it.we, *Sg = (float *)it.s;
    unsigned short *ID = (unsigned short *)it.id;
    for (int i = tid; i < nrows; i += nthr) {
        const long long k0 = v.row_ptr[row_g0 + row0 + i] - sbase, k1 = v.row_ptr[row_g0 + row0 + i + 1] - sbase;
        int m1 = 0, m2 = 0;
        for (long long k = k0; k < k1; ++k) {
            const uint32_t code = gcode[k];
            const bool sec = HAS2 && second_order(stab, code);
            const long long p = sec ? item_slot(it.ib2[i], m2++, K, it.n2, K * it.n1)
                                    : item_slot(it.ib1[i], m1++, K, it.n1, 0);
            const float w = gw[k];
            R[p] = gr[k];
            W[p] = w;
            WE[p] = w * stab[(code >> 24) * 9 + SP_E];
            ID[p] = (unsigned short)(code & 0xFFFFFFu);
            if (HAS2 && sec) Sg[p] = gs[k];
        }
    }
    __syncthreads();
}

// Write the owned synapses back to the global CSR arrays, applying the last
// step's gate map (fin.r: r-map, fin.s: s-map, by coefficient index).
template <bool HAS2, class Fin>
__device__ void store_items(const Items &it, const NetView &v, long long row_g0, long long sbase, int row0,
                            float *gr, float *gs, const uint32_t *gcode, const float *stab, const Fin &fin) {
    const int tid = threadIdx.x, nthr = blockDim.x, K = it.K;
    const float *R = (const float *)it.r, *Sg = (const float *)it.s;
    for (int i = tid; i < it.nrows; i += nthr) {
        const long long k0 = v.row_ptr[row_g0 + row0 + i] - sbase, k1 = v.row_ptr[row_g0 + row0 + i + 1] - sbase;
        int m1 = 0, m2 = 0;
        for (long long k = k0; k < k1; ++k) {
            const uint32_t code = gcode[k];
            const int ci = (int)(code & 0xFFFFFFu);
            const bool sec = HAS2 && second_order(stab, code);
            const long long p = sec ? item_slot(it.ib2[i], m2++, K, it.n2, K * it.n1)
                                    : item_slot(it.ib1[i], m1++, K, it.n1, 0);
            const float r0 = R[p];
            gr[k] = map_r(fin.r(ci), r0);
            if (HAS2 && sec) gs[k] = map_s(fin.s(ci), r0, Sg[p]);
        }
    }
}

// One synapse of the current stage: gate value from the affine map, then
// accumulate A += w G, B += wE G.  At the step's first stage the previous
// step's final map is applied and the new step-start gate stored.
__device__ __forceinline__ void syn1(bool first, float &r, float w, float we, float2 F, float &A, float &B) {
    const float g = map_r(F, r);
    if (first) r = g;
    A = fmaf(w, g, A);
    B = fmaf(we, g, B);
}

__device__ __forceinline__ void syn2(bool first, float &r, float &s, float w, float we, float2 F, float4 F2,
                                     float &A, float &B) {
    const float rr = map_r(F, r);
    const float ss = map_s(F2, r, s);
    if (first) {
        r = rr;
        s = ss;
    }
    const float s2 = ss * ss, s4 = s2 * s2;
    const float g = __fdiv_rn(s4, __fadd_rn(s4, F2.w));  // no contraction into an FMA: same bits everywhere
    A = fmaf(w, g, A);
    B = fmaf(we, g, B);
}

// Stage kinds ST: 0..3 the stages of classic RK4, 4 the single stage of
// forward Euler (first and last stage of its step), and 4 (n + 1) + s
// (8..23) stage s of an n-stage tableau (PSST_METHOD_TABLEAU), whose
// coefficients are read at run time.
__host__ __device__ constexpr bool stage_first(int ST) { return ST >= 8 ? (ST & 3) == 0 : (ST == 0 || ST == 4); }
__host__ __device__ constexpr bool stage_last(int ST) { return ST >= 8 ? (ST & 3) == (ST >> 2) - 2 : ST >= 3; }
__host__ __device__ constexpr int tableau_stage(int n, int s) { return 4 * (n + 1) + s; }

// Coefficients of stage ST: w, the weight of its slope in the step's sum
// (relative to the first nonzero weight); cn = dt a_{s+1}, the factor of the
// slope in the next stage's start; fin = dt times the scale of the sum at
// the step's end.  RK4: w = 1, 2, 2, 1, cn = dt/2, dt/2, dt, fin = dt/6.
struct StageCoef {
    float w, cn, fin;
};

template <int ST>
__device__ __forceinline__ StageCoef stage_coef(const NetView &v, float dt) {
    StageCoef c;
    if (ST >= 8) {
        constexpr int s = ST & 3;
        c.w = v.rk_w[s];
        c.cn = s < 3 ? v.rk_c[s < 3 ? s : 0] * dt : 0.0f;
        c.fin = v.rk_beta * dt;
    } else {
        c.w = (ST == 1 || ST == 2) ? 2.0f : 1.0f;
        c.cn = (ST == 2) ? dt : 0.5f * dt;
        c.fin = ST == 4 ? dt : dt * (1.0f / 6.0f);
    }
    return c;
}

// Stage descriptors: whether the stage is its step's first and last, its
// coefficients, and the first stage's term of the step's sum.  StageCT<ST>
// fixes the kind at compile time (kernels unrolled per stage kind);
// StageRT carries it at run time, so that one copy of the stage code serves
// every stage of every method (the classic RK4 and Euler stages as the
// tableau stages with the same coefficients: their first weight is 1, and
// 1 * d is d, so both descriptors give the same bits).
template <int ST>
struct StageCT {
    static constexpr bool first = stage_first(ST), last = stage_last(ST);
    StageCoef c;
    __device__ __forceinline__ float first_term(float d) const { return ST >= 8 ? __fmul_rn(c.w, d) : d; }
};

struct StageRT {
    bool first, last;
    StageCoef c;
    __device__ __forceinline__ float first_term(float d) const { return __fmul_rn(c.w, d); }
};

// Stages per step of the handle's method.
__host__ __device__ inline int method_stages(const NetView &v) {
    return v.method == PSST_METHOD_EULER ? 1 : v.method == PSST_METHOD_TABLEAU ? v.rk_ns : 4;
}

// Stage s of the handle's method at run time, with the coefficients
// stage_coef gives the corresponding compile-time kind.
__device__ __forceinline__ StageRT stage_rt(const NetView &v, int s, float dt) {
    StageRT r;
    const int ns = method_stages(v);
    r.first = s == 0;
    r.last = s == ns - 1;
    if (v.method == PSST_METHOD_TABLEAU) {
        r.c.w = v.rk_w[s];
        r.c.cn = s < 3 ? v.rk_c[s < 3 ? s : 0] * dt : 0.0f;
        r.c.fin = v.rk_beta * dt;
    } else {
        const bool euler = v.method == PSST_METHOD_EULER;
        r.c.w = (!euler && (s == 1 || s == 2)) ? 2.0f : 1.0f;
        r.c.cn = (!euler && s == 2) ? dt : 0.5f * dt;
        r.c.fin = euler ? dt : dt * (1.0f / 6.0f);
    }
    return r;
}

// S-phase: every item's partial sums (A, B) at stage ST.  Coef supplies
// r(ci) (float2 r-map) and s(ci) (float4 s-map, w = Kd).
template <bool HAS2, class Coef>
__device__ __forceinline__ void sphase(bool FIRST, const Items &it, const Coef &cf) {
    const int tid = threadIdx.x, nthr = blockDim.x, K = it.K, n1 = it.n1;
    for (int t = tid; t < n1; t += nthr) {
        float A = 0.0f, B = 0.0f;
        for (int j = 0; j < K; ++j) {
            const int c = j * n1 + t;
            float4 r = it.r[c];
            const float4 w = it.w[c], we = it.we[c];
            const ushort4 id = it.id[c];
            syn1(FIRST, r.x, w.x, we.x, cf.r(id.x), A, B);
            syn1(FIRST, r.y, w.y, we.y, cf.r(id.y), A, B);
            syn1(FIRST, r.z, w.z, we.z, cf.r(id.z), A, B);
            syn1(FIRST, r.w, w.w, we.w, cf.r(id.w), A, B);
            if (FIRST) it.r[c] = r;
        }
        it.pa[t] = A;
        it.pb[t] = B;
    }
    if (HAS2) {
        const int n2 = it.n2, base = K * n1;
        for (int t = tid; t < n2; t += nthr) {
            float A = 0.0f, B = 0.0f;
            for (int j = 0; j < K; ++j) {
                const int c = base + j * n2 + t;
                float4 r = it.r[c], s = it.s[c];
                const float4 w = it.w[c], we = it.we[c];
                const ushort4 id = it.id[c];
                syn2(FIRST, r.x, s.x, w.x, we.x, cf.r(id.x), cf.s(id.x), A, B);
                syn2(FIRST, r.y, s.y, w.y, we.y, cf.r(id.y), cf.s(id.y), A, B);
                syn2(FIRST, r.z, s.z, w.z, we.z, cf.r(id.z), cf.s(id.z), A, B);
                syn2(FIRST, r.w, s.w, w.w, we.w, cf.r(id.w), cf.s(id.w), A, B);
                if (FIRST) {
                    it.r[c] = r;
                    it.s[c] = s;
                }
            }
            it.pa[n1 + t] = A;
            it.pb[n1 + t] = B;
        }
    }
}

// Synaptic current of owned row i from its items' partials (fixed order).
template <bool HAS2>
__device__ __forceinline__ float row_current(const Items &it, int i, float V) {
    float A = 0.0f, B = 0.0f;
    for (int t = it.ib1[i]; t < it.ib1[i + 1]; ++t) {
        A += it.pa[t];
        B += it.pb[t];
    }
    if (HAS2)
        for (int t = it.ib2[i]; t < it.ib2[i + 1]; ++t) {
            A += it.pa[it.n1 + t];
            B += it.pb[it.n1 + t];
        }
    return fmaf(V, A, -B);
}

// ------------------------------------------------- per-pair gate variant
//
// When all gates of a (presynaptic neuron, type) pair hold the same value
// (true from rest, and preserved by the dynamics), each stage's gate value
// is computed once per pair, G_p = P_s + Q_s r0_p with the same operations
// as the per-synapse path, and the items carry no gate state.  A row's
// synapses are then cut into items per synapse type, so that an item needs
// only A = sum w G (the reversal potential E is the item's, not the
// synapse's): chunk = float4 w + ushort4 gate-table index, one partial per
// item, and I_syn,i = V_i sum_t A_t - sum_t E_t A_t over the row's items in
// item order (bitwise reproducible for a given K).

__host__ __device__ inline long long items_smem_bytes_pair(int n_items, int K, int nrows) {
    const long long c = (long long)K * n_items;
    return c * (16 + 8) + 8LL * n_items + 4LL * (nrows + 1) + 64;
}

__device__ inline Items carve_items_pair(unsigned char *base, int nrows, int K, int n_items) {
    Items it;
    it.nrows = nrows;
    it.K = K;
    it.n1 = n_items;
    it.n2 = 0;
    const long long c = (long long)K * n_items;
    unsigned char *p = base;
    it.r = nullptr;
    it.s = nullptr;
    it.we = nullptr;
    it.w = (float4 *)p;
    p += 16 * c;
    it.id = (ushort4 *)p;
    p += 8 * c;
    it.pa = (float *)p;   // item partial A
    p += 4LL * n_items;
    it.pb = (float *)p;   // item's reversal potential E
    p += 4LL * n_items;
    it.ib1 = (int *)p;
    it.ib2 = nullptr;
    return it;
}

// Synapses of a row part of one type in items of K chunks.
__host__ __device__ inline int typed_row_items(const int *cnt, int nt, int K) {
    int n = 0;
    for (int t = 0; t < nt; ++t) n += part_items(cnt[t], K);
    return n;
}

// Items of rows [row0, row0 + nrows), per row one run of items per synapse
// type (types in increasing order); the gate-table index of a synapse is its
// (neuron, type) pair index, or tix[pair] when a compact table of the used
// pairs is given.  tmp: shared scratch of nrows + 1 ints.
__device__ inline void load_items_pair(Items &it, const NetView &v, long long row_g0, long long sbase, int row0,
                                const float *gw, const uint32_t *gcode, const float *stab, int *tmp,
                                const int *tix) {
    const int tid = threadIdx.x, nthr = blockDim.x, nrows = it.nrows, K = it.K, nt = v.n_stypes;
    for (int i = tid; i < nrows; i += nthr) {
        const long long k0 = v.row_ptr[row_g0 + row0 + i] - sbase, k1 = v.row_ptr[row_g0 + row0 + i + 1] - sbase;
        int cnt[PSST_MAX_SYN_TYPES] = {};
        for (long long k = k0; k < k1; ++k) ++cnt[gcode[k] >> 24];
        tmp[i] = typed_row_items(cnt, nt, K);
    }
    __syncthreads();
    block_scan(tmp, it.ib1, nrows);
    const long long chunks = (long long)K * it.n1;
    for (long long c = tid; c < chunks; c += nthr) {
        it.w[c] = make_float4(0.f, 0.f, 0.f, 0.f);
        it.id[c] = make_ushort4(0, 0, 0, 0);
    }
    __syncthreads();
    float *W = (float *)it.w;
    unsigned short *ID = (unsigned short *)it.id;
    for (int i = tid; i < nrows; i += nthr) {
        const long long k0 = v.row_ptr[row_g0 + row0 + i] - sbase, k1 = v.row_ptr[row_g0 + row0 + i + 1] - sbase;
        int cnt[PSST_MAX_SYN_TYPES] = {}, base[PSST_MAX_SYN_TYPES], m[PSST_MAX_SYN_TYPES] = {};
        for (long long k = k0; k < k1; ++k) ++cnt[gcode[k] >> 24];
        int b = it.ib1[i];
        for (int t = 0; t < nt; ++t) {
            base[t] = b;
            const int q = part_items(cnt[t], K);
            for (int u = 0; u < q; ++u) it.pb[b + u] = stab[t * 9 + SP_E];
            b += q;
        }
        for (long long k = k0; k < k1; ++k) {
            const uint32_t code = gcode[k];
            const int t = (int)(code >> 24);
            const long long p = item_slot(base[t], m[t]++, K, it.n1, 0);
            const uint32_t ci = code & 0xFFFFFFu;
            W[p] = gw[k];
            ID[p] = (unsigned short)(tix ? tix[ci] : (int)ci);
        }
    }
    __syncthreads();
}

// S-phase of the per-pair variant: every item's A = sum w G with G the gate
// of entry id.  The gate table holds 2^lrep copies of each entry side by
// side (entry e, copy c at e * 2^lrep + c) and lane l reads copy
// l mod 2^lrep: with 32 copies the 32 lanes of a gather hit 32 different
// banks whatever the entries.
// sphase_pair_range: the items [t0, t1) by the threads j = 0..nthr-1 of a
// group (thread j takes items t0 + j, t0 + j + nthr, ...).
__device__ __forceinline__ void sphase_pair_range(const Items &it, const float *Gt, int lrep, int t0, int t1, int j,
                                                  int nthr) {
    const int K = it.K, n = it.n1;
    const float *Gl = Gt + (threadIdx.x & ((1 << lrep) - 1));
    for (int t = t0 + j; t < t1; t += nthr) {
        float A = 0.0f;
#pragma unroll 4
        for (int j = 0; j < K; ++j) {  // unrolled: several chunks' loads in flight, sums in order
            const int c = j * n + t;
            const float4 w = it.w[c];
            const ushort4 id = it.id[c];
            const float g0 = Gl[id.x << lrep], g1 = Gl[id.y << lrep], g2 = Gl[id.z << lrep], g3 = Gl[id.w << lrep];
            A = fmaf(w.x, g0, A);
            A = fmaf(w.y, g1, A);
            A = fmaf(w.z, g2, A);
            A = fmaf(w.w, g3, A);
        }
        it.pa[t] = A;
    }
}

__device__ __forceinline__ void sphase_pair(const Items &it, const float *Gt, int lrep) {
    sphase_pair_range(it, Gt, lrep, 0, it.n1, threadIdx.x, blockDim.x);
}

// Synaptic current of owned row i from its typed items (fixed order).
// Called by all 32 lanes of a warp (valid = false: a lane without a row,
// which sums nothing): the item partials are loaded in blocks of 8 with
// predication, over the warp's largest item count, so the loop is uniform
// across the warp (a divergent, data-dependent loop costs several times its
// loads and adds here).  The sums run in item order as
// A += a_t, B = fma(E_t, a_t, B); the padding adds exact zeros (A and B are
// never -0: A sums w G >= 0 terms, B starts at +0), so every path gets the
// same bits as the plain item-order loop.
__device__ __forceinline__ float row_current_pair(const Items &it, int i, float V, bool valid = true) {
    const int t0 = valid ? it.ib1[i] : 0;
    const int n = valid ? it.ib1[i + 1] - t0 : 0;
    const int nmax = __reduce_max_sync(0xffffffffu, (unsigned)n);
    float A = 0.0f, B = 0.0f;
    for (int base = 0; base < nmax; base += 8) {
        float a[8], e[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const bool in = base + q < n;
            a[q] = in ? it.pa[t0 + base + q] : 0.0f;
            e[q] = in ? it.pb[t0 + base + q] : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            A += a[q];
            B = fmaf(e[q], a[q], B);
        }
    }
    return fmaf(V, A, -B);
}

// Store the gate of entry e in all 2^lrep copies (16-byte stores from 4
// copies on, the lane's first store rotated so that a warp's stores spread
// over the banks).
__device__ __forceinline__ void put_gate(float *Gt, int e, int lrep, float G) {
    const int R = 1 << lrep, l = (int)threadIdx.x;
    float *row = Gt + ((long long)e << lrep);
    if (R >= 4) {
        // up to 8 predicated 16-byte stores, no loop (R <= 32)
        const float4 g4 = make_float4(G, G, G, G);
        const int n4 = R >> 2;
#pragma unroll
        for (int c = 0; c < 8; ++c)
            if (c < n4) ((float4 *)row)[(c + l) & (n4 - 1)] = g4;
    } else {
        row[0] = G;
        if (R > 1) row[1] = G;
    }
}

// Gate value G of a pair from its stage maps and step-start gates, with
// exactly the operations of syn1/syn2 (first order: r; second order:
// s^4 / (s^4 + Kd), Kd in F2.w).
__device__ __forceinline__ float pair_gate(bool second, float2 F, float4 F2, float r0, float s0, float r0lo,
                                           float s0lo) {
    const float rr = __fadd_rn(r0, __fadd_rn(fmaf(F.y, r0, F.x), r0lo));
    if (!second) return rr;
    const float ss = __fadd_rn(s0, __fadd_rn(fmaf(F2.z, s0, fmaf(F2.y, r0, F2.x)), s0lo));
    const float s2 = ss * ss, s4 = s2 * s2;
    return __fdiv_rn(s4, __fadd_rn(s4, F2.w));
}

// A pair's step-start gates (r0, s0) with their remainders advanced by the
// step's final maps (F, F2).
__device__ __forceinline__ void pair_step(bool second, float2 F, float4 F2, float &r0, float &s0, float &r0lo,
                                          float &s0lo) {
    const float r_old = r0;
    ext_add(r0, r0lo, fmaf(F.y, r_old, F.x));
    if (second) ext_add(s0, s0lo, fmaf(F2.z, s0, fmaf(F2.y, r_old, F2.x)));
}

// Gate-map update of one (presynaptic neuron j, synapse type tau) pair at
// stage ST from the stage-ST potential V of j.  cur/acc hold this stage's
// map and the running RK4 sum; writes the next stage's map into cur, or at
// the step's last stage the step's final map into fin.  The s-map's fourth
// component carries Kd (1 for first-order types, whose s-map is never used).
template <bool HAS2, class SG>
__device__ __forceinline__ void coef_update(const float *sp, float V, const SG &sg, float2 &cur, float2 &acc,
                                            float2 &fin, float4 &cur2, float4 &acc2, float4 &fin2) {
    const bool FIRST = sg.first, LAST = sg.last;
    const float WGT = sg.c.w, cnext = sg.c.cn, dt6 = sg.c.fin;
    const float T = transmitter(V, sp[SP_VP], sp[SP_KP]);  // table holds 1/Kp
    // explicit roundings: no product is contracted into an FMA or folded
    // with a constant stage weight, so every kernel and stage kind (constant
    // or run-time coefficients) gets the same bits
    const float a_ = __fmul_rn(sp[SP_A], T), bb = __fadd_rn(a_, sp[SP_B]);
    // stage map (P, Qm) and (U, X, Zm) in increment form (Q = 1 + Qm, Z = 1 + Zm);
    // the first stage's is the identity
    float P = 0.0f, Qm = 0.0f, U = 0.0f, X = 0.0f, Zm = 0.0f;
    if (!FIRST) {
        P = cur.x;
        Qm = cur.y;
        if (HAS2) {
            U = cur2.x;
            X = cur2.y;
            Zm = cur2.z;
        }
    }
    // slope a T (1 - r) - b r = kP + kQ r0, with kQ = -bb Q = -bb - bb Qm
    const float kP = fmaf(-bb, P, a_), kQ = fmaf(-bb, Qm, -bb);
    float2 A1 = make_float2(sg.first_term(kP), sg.first_term(kQ));
    if (!FIRST) A1 = make_float2(fmaf(WGT, kP, acc.x), fmaf(WGT, kQ, acc.y));
    if (!LAST) {
        acc = A1;
        cur = make_float2(cnext * kP, cnext * kQ);
    } else {
        fin = make_float2(dt6 * A1.x, dt6 * A1.y);
    }
    if (HAS2) {
        const float K3 = sp[SP_K3], K4 = sp[SP_K4];
        const float Kd = sp[SP_KIND] != 0.0f ? sp[SP_KD] : 1.0f;
        // slope K3 r - K4 s = kU + kX r0 + kZ s0 with kX = K3 Q - K4 X, kZ = -K4 Z
        const float kU = fmaf(K3, P, __fmul_rn(-K4, U)), kX = fmaf(K3, Qm, fmaf(-K4, X, K3));
        const float kZ = fmaf(-K4, Zm, -K4);
        float4 A2 = make_float4(sg.first_term(kU), sg.first_term(kX), sg.first_term(kZ), 0.0f);
        if (!FIRST) A2 = make_float4(fmaf(WGT, kU, acc2.x), fmaf(WGT, kX, acc2.y), fmaf(WGT, kZ, acc2.z), 0.0f);
        if (!LAST) {
            acc2 = A2;
            cur2 = make_float4(cnext * kU, cnext * kX, cnext * kZ, Kd);
        } else {
            fin2 = make_float4(dt6 * A2.x, dt6 * A2.y, dt6 * A2.z, Kd);
        }
    }
}

// Right-hand side and stage update of owned neuron i at stage ST, in two
// independent halves run by different threads: the potential (synaptic and
// ionic currents) and the gates m, h, n (rate functions).  y0/acc hold
// [4][n] (V, m, h, n); the stage gates are double-buffered by stage parity,
// ysc = [3][n] of this stage (read by both halves), ysn = [3][n] of the next.

// Potential, in two parts so that everything independent of the synaptic
// current (the ionic currents, the loads of the RK4 sums) is issued before
// the row's item partials are summed: neuron_v_pre, then neuron_v_post,
// which returns the next stage's V, or after the step's last stage (ST 3, or
// 4 for Euler) the new step-start V.
struct VPre {
    float ie;    // I_ext - I_ion
    float invC;  // 1 / C
    float y0;    // step-start V
    float lo;    // its remainder (compensated state)
    float acc;   // RK4 sum of V's stage slopes so far
};

template <class SG>
__device__ __forceinline__ VPre neuron_v_pre(const SG &sg, int i, int n, float V, const float *ysc,
                                             const float *y0, const float *ylo, const float *acc, const float *prm,
                                             float iext) {
    const bool FIRST = sg.first;
    const float m = ysc[i], h = ysc[n + i], nn = ysc[2 * n + i];
    // explicit roundings (no contraction left to the compiler), so that every
    // kernel evaluates the same operations in whatever context it is inlined
    const float m3h = __fmul_rn(__fmul_rn(__fmul_rn(m, m), m), h);
    const float n2 = __fmul_rn(nn, nn), n4 = __fmul_rn(n2, n2);
    float iion = __fmul_rn(__fmul_rn(prm[NP_GNA * n + i], m3h), __fsub_rn(V, prm[NP_ENA * n + i]));
    iion = fmaf(__fmul_rn(prm[NP_GK * n + i], n4), __fsub_rn(V, prm[NP_EK * n + i]), iion);
    iion = fmaf(prm[NP_GL * n + i], __fsub_rn(V, prm[NP_EL * n + i]), iion);
    iion = fmaf(prm[NP_GKL * n + i], __fsub_rn(V, prm[NP_EKL * n + i]), iion);
    VPre r;
    r.ie = __fsub_rn(iext, iion);
    r.invC = prm[NP_C * n + i];  // prm row 0 holds 1/C
    r.y0 = y0[i];
    r.lo = ylo[i];
    r.acc = FIRST ? 0.0f : acc[i];
    return r;
}

template <class SG>
__device__ __forceinline__ float neuron_v_post(const SG &sg, int i, const VPre &p, float isyn, float *y0,
                                              float *ylo, float *acc) {
    const bool FIRST = sg.first, LAST = sg.last;
    const float WGT = sg.c.w, cnext = sg.c.cn, dt6 = sg.c.fin;
    const float d = __fmul_rn(__fsub_rn(p.ie, isyn), p.invC);
    const float ac = FIRST ? sg.first_term(d) : fmaf(WGT, d, p.acc);
    if (!LAST) {
        acc[i] = ac;
        return ext_stage(p.y0, p.lo, cnext, d);
    }
    float hi = p.y0, lo = p.lo;
    ext_step(hi, lo, dt6, ac);
    y0[i] = hi;
    ylo[i] = lo;
    return hi;
}

template <class SG>
__device__ __forceinline__ float neuron_v(const SG &sg, int i, int n, float V, const float *ysc, float *y0,
                                          float *ylo, float *acc, const float *prm, float iext, float isyn) {
    return neuron_v_post(sg, i, neuron_v_pre(sg, i, n, V, ysc, y0, ylo, acc, prm, iext), isyn, y0, ylo, acc);
}

// Gates: writes the next stage's m, h, n, or after the last stage the new
// step-start ones.
template <class SG>
__device__ __forceinline__ void neuron_gates(const SG &sg, int i, int n, float V, const float *ysc, float *ysn,
                                             float *y0, float *ylo, float *acc) {
    const bool FIRST = sg.first, LAST = sg.last;
    const float WGT = sg.c.w, cnext = sg.c.cn, dt6 = sg.c.fin;
    const float m = ysc[i], h = ysc[n + i], nn = ysc[2 * n + i];
    const Rates q = hh_rates(V);
    float d[3];
    d[0] = fmaf(q.am, __fsub_rn(1.0f, m), -__fmul_rn(q.bm, m));
    d[1] = fmaf(q.ah, __fsub_rn(1.0f, h), -__fmul_rn(q.bh, h));
    d[2] = fmaf(q.an, __fsub_rn(1.0f, nn), -__fmul_rn(q.bn, nn));
#pragma unroll
    for (int x = 0; x < 3; ++x) {
        const int ix = (x + 1) * n + i;
        const float ac = FIRST ? sg.first_term(d[x]) : fmaf(WGT, d[x], acc[ix]);
        float yn;
        if (!LAST) {
            acc[ix] = ac;
            yn = ext_stage(y0[ix], ylo[ix], cnext, d[x]);
        } else {
            float hi = y0[ix], lo = ylo[ix];
            ext_step(hi, lo, dt6, ac);
            y0[ix] = hi;
            ylo[ix] = lo;
            yn = hi;
        }
        ysn[x * n + i] = yn;
    }
}

}  // namespace psst
