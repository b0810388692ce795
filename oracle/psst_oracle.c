/*
 * FP64 CPU oracle for RK4 integration of coupled Hodgkin-Huxley networks.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two meet only through
 * the seeded input arrays.
 *
 * What it computes (all plain loops, float64, no reordering):
 *   - the initial value problem dy/dt = f(y) of the paper's Eq. (ode), with
 *     y the vectorised network state X' = [V, m, h, n] of Sec. "Brain
 *     simulations as computational graphs", extended by one gate r (and s for
 *     second-order synapses) per synapse (Sec. "Circumventing memory
 *     constraints", item 1: synaptic variables stored sparsely);
 *   - the recursion X_{i+1} = F(X_i, t_i, eps_i) with eps_i read as the step
 *     dt and F the classic fourth-order Runge-Kutta map (Sec. "Brain
 *     simulations ...", RK4 paragraph) or forward Euler (Eq. euler);
 *   - the Philox4x32-10 counter-based generator of Salmon et al., SC'11,
 *     used for shot-noise input.
 *
 * The paper gives the HH model only by name and state vector; the rate
 * functions and constants are the textbook squid-axon set in the -65 mV
 * convention.  Synapses are kinetic gates driven by a sigmoidal transmitter
 * T(V_pre) = 1 / (1 + exp(-(V_pre - Vp) / Kp)).
 *
 * State layout (length 4N + 2S): V[N], m[N], h[N], n[N], r[S], s[S].
 * Parameter tables (row per type):
 *   neuron: C, gNa, gK, gL, ENa, EK, EL, gKL, EKL
 *   synapse: kind, a, b, K3, K4, Kd, E, Vp, Kp
 *     kind 0: dr/dt = a T (1-r) - b r,                   G = r
 *     kind 1: dr/dt = a T (1-r) - b r, ds/dt = K3 r - K4 s, G = s^4/(s^4+Kd)
 *   synaptic current into the postsynaptic neuron: w G (V_post - E).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { P_C, P_GNA, P_GK, P_GL, P_ENA, P_EK, P_EL, P_GKL, P_EKL, P_NCOL };
enum { Q_KIND, Q_A, Q_B, Q_K3, Q_K4, Q_KD, Q_E, Q_VP, Q_KP, Q_NCOL };

typedef struct {
    int64_t N, S;
    const int32_t *ntype;       /* [N] */
    const double *nparams;      /* [n_ntypes * P_NCOL] */
    const int64_t *row_ptr;     /* [N+1], CSR by postsynaptic neuron */
    const int64_t *pre;         /* [S], GLOBAL presynaptic neuron index */
    const double *w;            /* [S] */
    const int32_t *stype;       /* [S] */
    const double *sparams;      /* [n_stypes * Q_NCOL] */
    const double *i_const;      /* [N] */
    const double *pulse_amp;    /* [N] */
    const int64_t *pulse_on;    /* [N] (per neuron: its network's window) */
    const int64_t *pulse_off;   /* [N] */
    uint64_t noise_seed;
    uint32_t noise_thresh;
    double noise_amp;
    double dt;
} orc_net;

/* ---------------------------------------------------------------- Philox */

/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
   32x32->64 multiplies with the round keys advanced by Weyl increments. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* One noise draw for (step, neuron): counter (step_lo, step_hi, neuron, 0),
   key (seed_lo, seed_hi); the event test is on the top 24 bits of word 0. */
int orc_noise_event(uint64_t seed, uint32_t thresh, int64_t step, int64_t neuron)
{
    uint32_t ctr[4] = {(uint32_t)(uint64_t)step, (uint32_t)((uint64_t)step >> 32),
                       (uint32_t)neuron, 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return (out[0] >> 8) < thresh;
}

/* ------------------------------------------------------ HH rate functions */

/* u / (1 - exp(-u)), with its limit 1 at u = 0 */
static double ratio_u(double u)
{
    if (u == 0.0) return 1.0;
    return u / (-expm1(-u));
}

/* alpha_m, beta_m, alpha_h, beta_h, alpha_n, beta_n in 1/ms at V in mV */
void orc_rates(double V, double out[6])
{
    out[0] = ratio_u((V + 40.0) / 10.0);                 /* 0.1(V+40)/(1-e^{-(V+40)/10}) */
    out[1] = 4.0 * exp(-(V + 65.0) / 18.0);
    out[2] = 0.07 * exp(-(V + 65.0) / 20.0);
    out[3] = 1.0 / (1.0 + exp(-(V + 35.0) / 10.0));
    out[4] = 0.1 * ratio_u((V + 55.0) / 10.0);           /* 0.01(V+55)/(1-e^{-(V+55)/10}) */
    out[5] = 0.125 * exp(-(V + 65.0) / 80.0);
}

void orc_steady_gates(double V, double out[3])
{
    double r[6];
    orc_rates(V, r);
    out[0] = r[0] / (r[0] + r[1]);
    out[1] = r[2] / (r[2] + r[3]);
    out[2] = r[4] / (r[4] + r[5]);
}

double orc_transmitter(double V, double Vp, double Kp)
{
    return 1.0 / (1.0 + exp(-(V - Vp) / Kp));
}

/* ------------------------------------------------------------ input, RHS */

void orc_input(const orc_net *net, int64_t step, double *iext)
{
    for (int64_t i = 0; i < net->N; ++i) {
        double I = net->i_const[i];
        if (step >= net->pulse_on[i] && step < net->pulse_off[i]) I += net->pulse_amp[i];
        if (net->noise_thresh && orc_noise_event(net->noise_seed, net->noise_thresh, step, i))
            I += net->noise_amp;
        iext[i] = I;
    }
}

/* dy = f(y) for the whole network with the step's input current iext. */
void orc_rhs(const orc_net *net, const double *iext, const double *y, double *dy)
{
    const int64_t N = net->N, S = net->S;
    const double *V = y, *m = y + N, *h = y + 2 * N, *n = y + 3 * N;
    const double *r = y + 4 * N, *s = y + 4 * N + S;
    double *dV = dy, *dm = dy + N, *dh = dy + 2 * N, *dn = dy + 3 * N;
    double *dr = dy + 4 * N, *ds = dy + 4 * N + S;

    for (int64_t i = 0; i < N; ++i) {
        /* synaptic current onto i: brute-force sum over its CSR row */
        double isyn = 0.0;
        for (int64_t k = net->row_ptr[i]; k < net->row_ptr[i + 1]; ++k) {
            const double *q = net->sparams + (int64_t)net->stype[k] * Q_NCOL;
            int64_t j = net->pre[k];
            double T = orc_transmitter(V[j], q[Q_VP], q[Q_KP]);
            double G;
            dr[k] = q[Q_A] * T * (1.0 - r[k]) - q[Q_B] * r[k];
            if (q[Q_KIND] == 0.0) {
                ds[k] = 0.0;
                G = r[k];
            } else {
                ds[k] = q[Q_K3] * r[k] - q[Q_K4] * s[k];
                double s4 = s[k] * s[k] * s[k] * s[k];
                G = s4 / (s4 + q[Q_KD]);
            }
            isyn += net->w[k] * G * (V[i] - q[Q_E]);
        }
        const double *p = net->nparams + (int64_t)net->ntype[i] * P_NCOL;
        double a[6];
        orc_rates(V[i], a);
        double iNa = p[P_GNA] * m[i] * m[i] * m[i] * h[i] * (V[i] - p[P_ENA]);
        double iK = p[P_GK] * n[i] * n[i] * n[i] * n[i] * (V[i] - p[P_EK]);
        double iL = p[P_GL] * (V[i] - p[P_EL]);
        double iKL = p[P_GKL] * (V[i] - p[P_EKL]);
        dV[i] = (iext[i] - iNa - iK - iL - iKL - isyn) / p[P_C];
        dm[i] = a[0] * (1.0 - m[i]) - a[1] * m[i];
        dh[i] = a[2] * (1.0 - h[i]) - a[3] * h[i];
        dn[i] = a[4] * (1.0 - n[i]) - a[5] * n[i];
    }
}

/* ------------------------------------------------ generic explicit steppers */

typedef void (*rhs_fn)(void *ctx, const double *y, double *dy);

/* classic RK4: c = (0, 1/2, 1/2, 1), b = (1, 2, 2, 1)/6 */
static void rk4_step(int64_t d, double h, rhs_fn f, void *ctx, double *y, double *work)
{
    double *k1 = work, *k2 = work + d, *k3 = work + 2 * d, *k4 = work + 3 * d;
    double *Y = work + 4 * d;
    f(ctx, y, k1);
    for (int64_t i = 0; i < d; ++i) Y[i] = y[i] + 0.5 * h * k1[i];
    f(ctx, Y, k2);
    for (int64_t i = 0; i < d; ++i) Y[i] = y[i] + 0.5 * h * k2[i];
    f(ctx, Y, k3);
    for (int64_t i = 0; i < d; ++i) Y[i] = y[i] + h * k3[i];
    f(ctx, Y, k4);
    for (int64_t i = 0; i < d; ++i)
        y[i] = y[i] + h / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
}

/* forward Euler, Eq. (euler) */
static void euler_step(int64_t d, double h, rhs_fn f, void *ctx, double *y, double *work)
{
    f(ctx, y, work);
    for (int64_t i = 0; i < d; ++i) y[i] = y[i] + h * work[i];
}

static void take_step(int order, int64_t d, double h, rhs_fn f, void *ctx, double *y, double *work)
{
    if (order == 1) euler_step(d, h, f, ctx, y, work);
    else rk4_step(d, h, f, ctx, y, work);
}

/* ----------------------------------------------- linear ODE (driver check) */

typedef struct { int64_t d; const double *A; } lin_ctx;

static void lin_rhs(void *c, const double *y, double *dy)
{
    const lin_ctx *L = (const lin_ctx *)c;
    for (int64_t i = 0; i < L->d; ++i) {
        double acc = 0.0;
        for (int64_t j = 0; j < L->d; ++j) acc += L->A[i * L->d + j] * y[j];
        dy[i] = acc;
    }
}

/* dy/dt = A y, nsteps steps of size h, through the same stepper the network
   integration uses.  Returns 0, or -1 if out of memory. */
int orc_linear_integrate(int64_t d, const double *A, double *y, double h, int64_t nsteps, int order)
{
    double *work = (double *)malloc(sizeof(double) * 5 * (size_t)d);
    if (!work) return -1;
    lin_ctx c = {d, A};
    for (int64_t k = 0; k < nsteps; ++k) take_step(order, d, h, lin_rhs, &c, y, work);
    free(work);
    return 0;
}

/* ------------------------------------------------------ network integration */

typedef struct { const orc_net *net; const double *iext; } net_ctx;

static void net_rhs(void *c, const double *y, double *dy)
{
    const net_ctx *nc = (const net_ctx *)c;
    orc_rhs(nc->net, nc->iext, y, dy);
}

/* Integrate nsteps steps starting at global step index step0 (time
   t0 + step0*dt).  The input current of step k is held over its stages.
   After each step the global index k+1 is checked: if (k+1) % rec_stride == 0
   the membrane potentials are appended to rec ([frame][N]) while fewer than
   rec_cap frames have been written.  Returns the number of frames written,
   or -1 on allocation failure. */
int64_t orc_integrate(const orc_net *net, double *y, int64_t step0, int64_t nsteps, int order,
                      int64_t rec_stride, double *rec, int64_t rec_cap)
{
    const int64_t d = 4 * net->N + 2 * net->S;
    double *work = (double *)malloc(sizeof(double) * (5 * (size_t)d + (size_t)net->N + 1));
    if (!work) return -1;
    double *iext = work + 5 * d;
    net_ctx c = {net, iext};
    int64_t frames = 0;
    for (int64_t k = step0; k < step0 + nsteps; ++k) {
        orc_input(net, k, iext);
        take_step(order, d, net->dt, net_rhs, &c, y, work);
        if (rec_stride > 0 && (k + 1) % rec_stride == 0 && frames < rec_cap) {
            memcpy(rec + frames * net->N, y, sizeof(double) * (size_t)net->N);
            ++frames;
        }
    }
    free(work);
    return frames;
}
