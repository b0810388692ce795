// Device-side data view and model arithmetic shared by the CUDA kernels.
//
// Model (the paper gives the HH model only by name and state vector,
// Sec. "Brain simulations as computational graphs"; the equations are the
// textbook squid-axon set in the -65 mV convention):
//   C dV/dt = I_ext - gNa m^3 h (V-ENa) - gK n^4 (V-EK) - gL (V-EL)
//             - gKL (V-EKL) - I_syn
//   dx/dt  = alpha_x(V) (1-x) - beta_x(V) x,   x in {m, h, n}
//   synapse gate r (first order) or pair r, s (second order) per synapse,
//   driven by the presynaptic transmitter T(V_pre); I_syn = sum w G (V-E).
#pragma once

#include <cstdint>

#include "../../include/psst.h"

namespace psst {

// Device pointers and sizes of one batch of networks (see psst.h for the
// meaning of each array).  Passed by value to every kernel.
struct NetView {
    int n_nets;
    int n_stypes;
    long long N, S;
    const int *net_off;          // [n_nets+1]
    const long long *row_ptr;    // [N+1]
    const uint32_t *syn_code;    // [S]: (type << 24) | (pre_local * n_stypes + type)
    const float *weight;         // [S]
    const int *neuron_type;      // [N]
    const float *nparams;        // [n_ntypes * 9]
    const float *sparams;        // [n_stypes * 9]
    const float *i_const;        // [N]
    const float *pulse_amp;      // [N] or null
    const long long *pulse_on;   // [n_nets]
    const long long *pulse_off;  // [n_nets]
    unsigned long long noise_seed;
    uint32_t noise_thresh;
    float noise_amp;
    float dt;
    float *state;                // [4N + 2S]: V, m, h, n, r, s
    float *state_lo;             // [4N + 2S] remainders of the compensated step sums (same layout), or
                                 // null: a launch starts them at zero and does not keep them
    float *rec;                  // [rec_cap][N] ring of V frames, or null
    int rec_stride;
    long long rec_cap;
    const uint8_t *net_flags;    // [n_nets]: bit 0 = has second-order synapses
    int *err;                    // device error word (first error wins)
    // the (presynaptic neuron, type) pairs that have synapses, per network in
    // pair order: compact index t of local pair p at pair_tix[net_off[b] *
    // n_stypes + p] (-1: no synapse), local pair of t at pair_of[pair_off[b] + t]
    const int *pair_tix;         // [N * n_stypes] or null
    const int *pair_of;          // [used pairs of all networks]
    const int *pair_off;         // [n_nets + 1]
    int method;                  // PSST_METHOD_RK4, _EULER or _TABLEAU
    // PSST_METHOD_TABLEAU: stages, next-stage factors a_{s+1} (s < rk_ns - 1),
    // the step weights as w_s = b_s / rk_beta with rk_beta the first nonzero b
    int rk_ns;
    float rk_c[3], rk_w[4], rk_beta;
};

enum : uint8_t { NET_HAS2 = 1, NET_PAIR = 2 };  // NET_PAIR: all gates of each (pre, type) pair equal

// Extra device state of the grid-wide mode (one network over all SMs).
constexpr int GRID_FLAG_STRIDE = 16;  // 64-bit words between two CTAs' phase flags (one 128-byte line each)

struct GridView {
    float2 *c1;                  // [2][N * n_stypes] gate maps (r), double-buffered by stage parity
    float4 *c2;                  // [2][N * n_stypes] gate maps (s), second-order networks only
    unsigned long long *flag;    // [gridDim.x][GRID_FLAG_STRIDE] last phase each CTA has published (zeroed before each launch)
    const int *row_split;        // [gridDim.x + 1] first row owned by each CTA
    const int *items;            // [2][gridDim.x] first- and second-order work items of each CTA
    int K;                       // 4-synapse chunks per work item
    unsigned long long timeout_ns;  // limit of one barrier wait
    // one gate per used (presynaptic neuron, type) pair (all gates of a pair equal)
    int pair;                    // 1: per-pair gate tables below; 0: per-synapse gates
    int mt;                      // entries of one gate table (used pairs, padded to a multiple of 4)
    const int *tix;              // [N * n_stypes] table index of each pair, -1 when no synapse uses it
    const long long *rep;        // [used pairs] one synapse of each pair (holds the pair's gates)
    int used;                    // used pairs (entries of the gate table)
    int gts;                     // words of one gate table: used + one heartbeat per CTA
    unsigned long long *gt;      // [2][gts] tagged words: each used pair's gate for the next stage, then the
                                 // CTAs' heartbeats; double-buffered by stage parity
    float *r0g, *s0g;            // [used pairs] step-start gates handed to the synapses' owners at the end
    float *r0lg, *s0lg;          // [used pairs] their remainders (null with a null state_lo)
};

// Column indices of the parameter tables.
enum { NP_C = 0, NP_GNA, NP_GK, NP_GL, NP_ENA, NP_EK, NP_EL, NP_GKL, NP_EKL };
enum { SP_KIND = 0, SP_A, SP_B, SP_K3, SP_K4, SP_KD, SP_E, SP_VP, SP_KP };

// Device state of one adjoint launch (psst_adjoint): per-network work-item
// size, checkpoint and segment storage, gradient accumulators, outputs.
struct AdjView {
    const int *K;               // [n_nets] chunks per row item (forward CTA)
    const int *n_items;         // [n_nets] row items
    const int *KC;              // [n_nets] chunks per column item (sweeping CTA)
    const int *n_citems;        // [n_nets] column items
    const int *cib;             // first column item of each pair, [M + 1] per network at cib_off
    const long long *cib_off;   // [n_nets]
    const int *ck;              // per column slot: the network's synapse index (-1: padding), at cslot_off
    const unsigned short *crow; // per column slot: the synapse's row (postsynaptic neuron)
    const long long *cslot_off; // [n_nets] column-slot offset of each network (multiple of 4)
    int ckpt_every;
    const float *ck_full;       // full states [4N+2S] every ckpt_every steps, recorded by the forward kernel
    const float *ck_full_lo;    // their remainders (same layout)
    long long dim;              // 4N + 2S
    float *seg;                 // step states of the segment being swept
    const long long *seg_off;   // [n_nets]
    float4 *gpart;              // per-segment FP32 partial weight gradients, column-slot order (4 per chunk)
    double *gtot;               // FP64 totals, column-slot order
    const float *dLdV;          // [n_frames][N]
    int n_frames;
    float *grad_w;              // [S] output, CSR order
    double *gp_neuron;          // [N][9] per-neuron parameter gradients
    float *grad_y0;             // [4][N] output: adjoint of V, m, h, n at the start
};

#define PSST_MAX_CL 4

// Per-network plan of the CTA/cluster kernel: the rows owned by each CTA of
// the network's cluster, the work-item size K (4-synapse chunks per item)
// and each CTA's number of first- and second-order items.
struct NetPlan {
    int split[PSST_MAX_CL + 1];
    int K;
    int n1[PSST_MAX_CL];
    int n2[PSST_MAX_CL];
    int lrep;  // per-pair gates: the gate table is held in 2^lrep copies (lane l reads copy l mod 2^lrep)
};

// Shared-memory layout of one CTA: its own neurons (n_own), the stage
// potential of every neuron it needs (n_all), the gate maps of m
// (neuron, type) pairs, then the synapse work items.  Computed the same way
// on host (sizing) and device (addressing).  Offsets in bytes, 16-aligned.
struct NeuronLayout {
    int cur2, acc2, fin2;  // float4 [m]: s-maps (second order only)
    int cur1, acc1, fin1;  // float2 [m]: r-maps
    int y0, ys, acc;       // float [4][n_own] step-start state, [2][3][n_own] stage m/h/n, [4][n_own] RK4 k-sum
    int ylo;               // float [4][n_own] remainders of the step-start state (compensated sums)
    int prm;               // float [9][n_own]: 1/C, gNa, gK, gL, ENa, EK, EL, gKL, EKL
    int iext;              // float [n_own]
    int inp;               // float [2][n_own]: constant current, pulse amplitude
    int vst;               // float [2][n_all]: stage potential, by stage parity
    int tmp;               // int [2][n_own + 1]: scan scratch
    int pair;              // per-pair variant: float [4][m] step-start r, s and their remainders,
                           // uint [m] presynaptic neuron << 8 | synapse type of each entry
    int gt;                // per-pair variant: float [m][rep] stage gate of each entry, rep copies
    int syn;               // start of the synapse items
};

__host__ __device__ inline int lay_take(int &o, long long bytes) {
    int at = o;
    o += (int)((bytes + 15) & ~15LL);
    return at;
}

__host__ __device__ inline NeuronLayout make_nlayout(int n_own, int n_all, int m, bool has2, bool pair = false,
                                                     int rep = 1) {
    NeuronLayout L;
    int o = 0;
    L.cur2 = has2 ? lay_take(o, 16LL * m) : -1;
    L.acc2 = has2 ? lay_take(o, 16LL * m) : -1;
    L.fin2 = has2 ? lay_take(o, 16LL * m) : -1;
    L.cur1 = lay_take(o, 8LL * m);
    L.acc1 = lay_take(o, 8LL * m);
    L.fin1 = lay_take(o, 8LL * m);
    // the stage potentials sit at the same offset in every CTA of a cluster
    // (peers write into them through distributed shared memory)
    L.vst = lay_take(o, 8LL * n_all);
    L.y0 = lay_take(o, 16LL * n_own);
    L.ylo = lay_take(o, 16LL * n_own);
    L.ys = lay_take(o, 24LL * n_own);  // stage m, h, n: [2][3][n] by stage parity
    L.acc = lay_take(o, 16LL * n_own);
    L.prm = lay_take(o, 36LL * n_own);
    L.iext = lay_take(o, 4LL * n_own);
    L.inp = lay_take(o, 8LL * n_own);
    L.tmp = lay_take(o, 8LL * (n_own + 1));
    L.pair = pair ? lay_take(o, 20LL * m) : -1;  // r0, s0, their remainders (float), neuron and type (uint)
    L.gt = pair ? lay_take(o, 4LL * rep * m) : -1;
    L.syn = o;
    return L;
}

// ---------------------------------------------------------------- maths

// u / (1 - exp(-u)); the removable singularity at u = 0 (alpha_m at -40 mV,
// alpha_n at -55 mV) is evaluated by its Bernoulli series for |u| < 0.1,
// where the FP32 difference 1 - exp(-u) would cancel.
__device__ __forceinline__ float ratio_u(float u) {
    if (fabsf(u) < 0.1f) {
        const float u2 = u * u;
        return fmaf(u2, fmaf(u2, -1.0f / 720.0f, 1.0f / 12.0f), fmaf(0.5f, u, 1.0f));
    }
    return __fdiv_rn(u, -expm1f(-u));
}

struct Rates {
    float am, bm, ah, bh, an, bn;
};

// Squid-axon rate functions (1/ms), V in mV, -65 mV rest convention.
__device__ __forceinline__ Rates hh_rates(float V) {
    Rates r;
    r.am = ratio_u((V + 40.0f) * 0.1f);
    r.bm = 4.0f * expf((V + 65.0f) * (-1.0f / 18.0f));
    r.ah = 0.07f * expf((V + 65.0f) * (-1.0f / 20.0f));
    r.bh = __frcp_rn(1.0f + expf((V + 35.0f) * (-0.1f)));
    r.an = 0.1f * ratio_u((V + 55.0f) * 0.1f);
    r.bn = 0.125f * expf((V + 65.0f) * (-1.0f / 80.0f));
    return r;
}

// Transmitter release T(V_pre) = 1 / (1 + exp(-(V - Vp) / Kp)).
__device__ __forceinline__ float transmitter(float V, float Vp, float inv_Kp) {
    return __frcp_rn(1.0f + expf((Vp - V) * inv_Kp));
}

// Philox4x32-10 (Salmon et al., SC'11), word 0 of the output block.
__device__ __forceinline__ uint32_t philox_word0(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    return c0;
}

// External current of global neuron gi during global step k, given its
// constant current, its pulse amplitude and whether step k lies inside its
// network's pulse window.
__device__ __forceinline__ float input_current(const NetView &v, float i_const, float pulse_amp, bool in_pulse,
                                               long long gi, long long k) {
    float I = i_const;
    if (in_pulse) I += pulse_amp;
    if (v.noise_thresh) {
        const uint32_t x = philox_word0((uint32_t)k, (uint32_t)((unsigned long long)k >> 32),
                                        (uint32_t)gi, 0u, (uint32_t)v.noise_seed,
                                        (uint32_t)(v.noise_seed >> 32));
        if ((x >> 8) < v.noise_thresh) I += v.noise_amp;
    }
    return I;
}

// Compensated state.  Within a launch, each step-start state variable is
// held as a pair (hi, lo): hi the FP32 value, lo the rounding remainder the
// step updates have accumulated, so that hi + lo carries about twice
// FP32's precision.  Rounding the small RK4 increment into an FP32 state
// every step otherwise dominates the drift of the FP32 trajectory from the
// exact map (it shifts spike times by microseconds over 10^4 steps).  A
// stage value is hi + (c d + lo); the step's update adds the increment with
// Knuth's TwoSum, which returns the rounded sum and its exact error.  All
// with explicit roundings, so every kernel computes the same bits.  A call
// starts with lo = 0 and returns hi: the FP32 state alone determines the
// continuation.
__device__ __forceinline__ float ext_stage(float hi, float lo, float c, float d) {
    return __fadd_rn(hi, fmaf(c, d, lo));
}

// (hi, lo) += c a: t = c a + lo, then TwoSum(hi, t).
__device__ __forceinline__ void ext_step(float &hi, float &lo, float c, float a) {
    const float t = fmaf(c, a, lo);
    const float s = __fadd_rn(hi, t);
    const float bp = __fsub_rn(s, hi);
    lo = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(t, bp));
    hi = s;
}

// (hi, lo) += inc (TwoSum of hi and inc + lo).
__device__ __forceinline__ void ext_add(float &hi, float &lo, float inc) { ext_step(hi, lo, 1.0f, inc); }

// Gate maps in increment form.  A stage's gate of a (presynaptic neuron,
// type) pair is an affine function of its step-start gates r0 (and s0):
//   r = r0 + (P + Qm r0),          (r-map F = (P, Qm))
//   s = s0 + (U + X r0 + Zm s0),   (s-map F2 = (U, X, Zm, Kd))
// i.e. Q = 1 + Qm and Z = 1 + Zm are kept as their differences from 1
// (rounding Q itself would cost bits of Qm, which is of order dt (a T + b)).
// The identity map is all zeros.
__device__ __forceinline__ float map_r(float2 F, float r0) { return __fadd_rn(r0, fmaf(F.y, r0, F.x)); }
__device__ __forceinline__ float map_s(float4 F2, float r0, float s0) {
    return __fadd_rn(s0, fmaf(F2.z, s0, fmaf(F2.y, r0, F2.x)));
}

__device__ __forceinline__ void set_error(int *err, int code) { atomicCAS(err, 0, code); }

}  // namespace psst
