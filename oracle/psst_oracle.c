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
 *     simulations ...", RK4 paragraph), forward Euler (Eq. euler), or an
 *     explicit Runge-Kutta map of a given tableau whose stage s uses only
 *     the slope of stage s-1 (the family both of the paper's methods
 *     belong to);
 *   - the Philox4x32-10 counter-based generator of Salmon et al., SC'11,
 *     used for shot-noise input;
 *   - the discrete adjoint (transpose) of each of these maps over the full
 *     per-synapse state, with the Jacobian-transpose products of the
 *     right-hand side derived by hand, giving gradients of a voltage-trace
 *     functional with respect to the initial state, the weights and the
 *     neuron-type parameters (checkpointed every K steps, recomputed).
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

/* Explicit Runge-Kutta map of a tableau whose only nonzero coupling
   coefficients are a_{s,s-1}.  tab = {n_stages (1..4), a_2, a_3, a_4,
   b_1, b_2, b_3, b_4}:
     Y_1 = y,  Y_s = y + h a_s k_{s-1},  k_s = f(Y_s),
     y_{n+1} = y + h sum_s b_s k_s. */
static void tab_step(const double *tab, int64_t d, double h, rhs_fn f, void *ctx, double *y, double *work)
{
    const int ns = (int)tab[0];
    double *k = work, *Y = work + d, *sum = work + 2 * d;
    for (int64_t i = 0; i < d; ++i) {
        Y[i] = y[i];
        sum[i] = 0.0;
    }
    for (int st = 1; st <= ns; ++st) {
        if (st > 1)
            for (int64_t i = 0; i < d; ++i) Y[i] = y[i] + h * tab[st - 1] * k[i];
        f(ctx, Y, k);
        for (int64_t i = 0; i < d; ++i) sum[i] += tab[3 + st] * k[i];
    }
    for (int64_t i = 0; i < d; ++i) y[i] = y[i] + h * sum[i];
}

/* order 4: classic RK4; order 1: forward Euler; order 0: the tableau tab */
static void take_step(int order, const double *tab, int64_t d, double h, rhs_fn f, void *ctx, double *y,
                      double *work)
{
    if (order == 0) tab_step(tab, d, h, f, ctx, y, work);
    else if (order == 1) euler_step(d, h, f, ctx, y, work);
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
int orc_linear_integrate(int64_t d, const double *A, double *y, double h, int64_t nsteps, int order,
                         const double *tab)
{
    double *work = (double *)malloc(sizeof(double) * 5 * (size_t)d);
    if (!work) return -1;
    lin_ctx c = {d, A};
    for (int64_t k = 0; k < nsteps; ++k) take_step(order, tab, d, h, lin_rhs, &c, y, work);
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
                      int64_t rec_stride, double *rec, int64_t rec_cap, const double *tab)
{
    const int64_t d = 4 * net->N + 2 * net->S;
    double *work = (double *)malloc(sizeof(double) * (5 * (size_t)d + (size_t)net->N + 1));
    if (!work) return -1;
    double *iext = work + 5 * d;
    net_ctx c = {net, iext};
    int64_t frames = 0;
    for (int64_t k = step0; k < step0 + nsteps; ++k) {
        orc_input(net, k, iext);
        take_step(order, tab, d, net->dt, net_rhs, &c, y, work);
        if (rec_stride > 0 && (k + 1) % rec_stride == 0 && frames < rec_cap) {
            memcpy(rec + frames * net->N, y, sizeof(double) * (size_t)net->N);
            ++frames;
        }
    }
    free(work);
    return frames;
}

/* ------------------------------------------------ discrete adjoint of RK4 */

/* d/du of u / (1 - exp(-u)); its limit at 0 is 1/2.  The Bernoulli series
   1/2 + u/6 - u^3/180 + u^5/5040 is used for |u| < 1e-2, where the closed
   form cancels. */
static double ratio_u_deriv(double u)
{
    if (fabs(u) < 1e-2) {
        double u2 = u * u;
        return 0.5 + u / 6.0 - u * u2 / 180.0 + u * u2 * u2 / 5040.0;
    }
    double e = exp(-u), den = -expm1(-u);
    return (den - u * e) / (den * den);
}

/* derivatives d/dV of alpha_m, beta_m, alpha_h, beta_h, alpha_n, beta_n */
void orc_rates_deriv(double V, double out[6])
{
    double r[6];
    orc_rates(V, r);
    out[0] = 0.1 * ratio_u_deriv((V + 40.0) / 10.0);
    out[1] = -r[1] / 18.0;
    out[2] = -r[2] / 20.0;
    out[3] = r[3] * (1.0 - r[3]) / 10.0;
    out[4] = 0.01 * ratio_u_deriv((V + 55.0) / 10.0);
    out[5] = -r[5] / 80.0;
}

/* Gradient accumulators of one adjoint run. */
typedef struct {
    double *gw;   /* [S] d/d weight */
    double *gnp;  /* [n_ntypes * P_NCOL] d/d neuron-type parameters */
} orc_grads;

/* u = J(y)^T v for the network right-hand side at state y (input iext), and
   params += (df/dtheta)^T v for the weights and the neuron-type parameters.
   Hand-derived from orc_rhs, term by term. */
void orc_vjp(const orc_net *net, const double *iext, const double *y, const double *v, double *u, orc_grads *g)
{
    const int64_t N = net->N, S = net->S;
    const double *V = y, *m = y + N, *h = y + 2 * N, *n = y + 3 * N;
    const double *r = y + 4 * N, *s = y + 4 * N + S;
    const double *vV = v, *vm = v + N, *vh = v + 2 * N, *vn = v + 3 * N;
    const double *vr = v + 4 * N, *vs = v + 4 * N + S;
    double *uV = u, *um = u + N, *uh = u + 2 * N, *un = u + 3 * N;
    double *ur = u + 4 * N, *us = u + 4 * N + S;

    for (int64_t i = 0; i < 4 * N + 2 * S; ++i) u[i] = 0.0;
    for (int64_t i = 0; i < N; ++i) {
        const double *p = net->nparams + (int64_t)net->ntype[i] * P_NCOL;
        double *gp = g ? g->gnp + (int64_t)net->ntype[i] * P_NCOL : NULL;
        const double q = vV[i] / p[P_C];  /* adjoint of dV/dt scaled by 1/C */
        double a[6], da[6];
        orc_rates(V[i], a);
        orc_rates_deriv(V[i], da);
        const double m3h = m[i] * m[i] * m[i] * h[i], n4 = n[i] * n[i] * n[i] * n[i];
        /* synaptic terms of the row: current, its V-derivative, weights, gates */
        double isyn = 0.0, gsum = 0.0;
        for (int64_t k = net->row_ptr[i]; k < net->row_ptr[i + 1]; ++k) {
            const double *sq = net->sparams + (int64_t)net->stype[k] * Q_NCOL;
            const double E = sq[Q_E];
            double G, dG;  /* gate and its derivative w.r.t. the variable it reads */
            if (sq[Q_KIND] == 0.0) {
                G = r[k];
                dG = 1.0;
                ur[k] += -q * net->w[k] * dG * (V[i] - E);
            } else {
                const double s4 = s[k] * s[k] * s[k] * s[k];
                G = s4 / (s4 + sq[Q_KD]);
                dG = 4.0 * s[k] * s[k] * s[k] * sq[Q_KD] / ((s4 + sq[Q_KD]) * (s4 + sq[Q_KD]));
                us[k] += -q * net->w[k] * dG * (V[i] - E);
            }
            isyn += net->w[k] * G * (V[i] - E);
            gsum += net->w[k] * G;
            if (g) g->gw[k] += -q * G * (V[i] - E);
        }
        const double iion = p[P_GNA] * m3h * (V[i] - p[P_ENA]) + p[P_GK] * n4 * (V[i] - p[P_EK]) +
                            p[P_GL] * (V[i] - p[P_EL]) + p[P_GKL] * (V[i] - p[P_EKL]);
        const double diion = p[P_GNA] * m3h + p[P_GK] * n4 + p[P_GL] + p[P_GKL];
        uV[i] += q * (-diion - gsum);
        uV[i] += vm[i] * (da[0] * (1.0 - m[i]) - da[1] * m[i]);
        uV[i] += vh[i] * (da[2] * (1.0 - h[i]) - da[3] * h[i]);
        uV[i] += vn[i] * (da[4] * (1.0 - n[i]) - da[5] * n[i]);
        um[i] += q * (-p[P_GNA] * 3.0 * m[i] * m[i] * h[i] * (V[i] - p[P_ENA])) - vm[i] * (a[0] + a[1]);
        uh[i] += q * (-p[P_GNA] * m[i] * m[i] * m[i] * (V[i] - p[P_ENA])) - vh[i] * (a[2] + a[3]);
        un[i] += q * (-p[P_GK] * 4.0 * n[i] * n[i] * n[i] * (V[i] - p[P_EK])) - vn[i] * (a[4] + a[5]);
        if (gp) {
            const double fV = (iext[i] - iion - isyn) / p[P_C];
            gp[P_C] += -q * fV;
            gp[P_GNA] += -q * m3h * (V[i] - p[P_ENA]);
            gp[P_GK] += -q * n4 * (V[i] - p[P_EK]);
            gp[P_GL] += -q * (V[i] - p[P_EL]);
            gp[P_GKL] += -q * (V[i] - p[P_EKL]);
            gp[P_ENA] += q * p[P_GNA] * m3h;
            gp[P_EK] += q * p[P_GK] * n4;
            gp[P_EL] += q * p[P_GL];
            gp[P_EKL] += q * p[P_GKL];
        }
    }
    /* gate equations: own-variable terms and the presynaptic voltage */
    for (int64_t k = 0; k < S; ++k) {
        const double *sq = net->sparams + (int64_t)net->stype[k] * Q_NCOL;
        const int64_t j = net->pre[k];
        const double T = orc_transmitter(V[j], sq[Q_VP], sq[Q_KP]);
        const double dT = T * (1.0 - T) / sq[Q_KP];
        ur[k] += -vr[k] * (sq[Q_A] * T + sq[Q_B]);
        uV[j] += vr[k] * sq[Q_A] * dT * (1.0 - r[k]);
        if (sq[Q_KIND] != 0.0) {
            ur[k] += vs[k] * sq[Q_K3];
            us[k] += -vs[k] * sq[Q_K4];
        }
    }
}

typedef void (*vjp_fn)(void *ctx, const double *y, const double *v, double *u);

/* Reverse of one classic RK4 step from y_n (Hager 2000; Sandu 2006): on
   entry lam holds the adjoint of y_{n+1}, on exit that of y_n.  With
   k_s = f(Y_s), the stage adjoints are
     kb4 = h/6 lam,           Yb4 = J(Y4)^T kb4
     kb3 = h/3 lam + h Yb4,   Yb3 = J(Y3)^T kb3
     kb2 = h/3 lam + h/2 Yb3, Yb2 = J(Y2)^T kb2
     kb1 = h/6 lam + h/2 Yb2, Yb1 = J(Y1)^T kb1
   and lam_n = lam + Yb1 + Yb2 + Yb3 + Yb4.  The vjp callback also adds the
   parameter terms (df/dtheta)^T kb_s. */
static void rk4_adjoint_step(int64_t d, double hstep, rhs_fn f, vjp_fn g, void *ctx, const double *y,
                             double *lam, double *work)
{
    double *Y1 = work, *Y2 = work + d, *Y3 = work + 2 * d, *Y4 = work + 3 * d;
    double *k = work + 4 * d, *kb = work + 5 * d, *Yb = work + 6 * d, *Ysum = work + 7 * d;
    for (int64_t i = 0; i < d; ++i) Y1[i] = y[i];
    f(ctx, Y1, k);
    for (int64_t i = 0; i < d; ++i) Y2[i] = y[i] + 0.5 * hstep * k[i];
    f(ctx, Y2, k);
    for (int64_t i = 0; i < d; ++i) Y3[i] = y[i] + 0.5 * hstep * k[i];
    f(ctx, Y3, k);
    for (int64_t i = 0; i < d; ++i) Y4[i] = y[i] + hstep * k[i];

    for (int64_t i = 0; i < d; ++i) kb[i] = hstep / 6.0 * lam[i];
    g(ctx, Y4, kb, Yb);
    for (int64_t i = 0; i < d; ++i) Ysum[i] = Yb[i];
    for (int64_t i = 0; i < d; ++i) kb[i] = hstep / 3.0 * lam[i] + hstep * Yb[i];
    g(ctx, Y3, kb, Yb);
    for (int64_t i = 0; i < d; ++i) Ysum[i] += Yb[i];
    for (int64_t i = 0; i < d; ++i) kb[i] = hstep / 3.0 * lam[i] + 0.5 * hstep * Yb[i];
    g(ctx, Y2, kb, Yb);
    for (int64_t i = 0; i < d; ++i) Ysum[i] += Yb[i];
    for (int64_t i = 0; i < d; ++i) kb[i] = hstep / 6.0 * lam[i] + 0.5 * hstep * Yb[i];
    g(ctx, Y1, kb, Yb);
    for (int64_t i = 0; i < d; ++i) lam[i] += Ysum[i] + Yb[i];
}

/* Reverse of one forward-Euler step, Eq. (euler): y_{n+1} = y_n + h f(y_n),
   so lam_n = lam + J(y_n)^T (h lam), with the parameter terms
   (df/dtheta)^T (h lam) added by the vjp callback. */
static void euler_adjoint_step(int64_t d, double hstep, vjp_fn g, void *ctx, const double *y, double *lam,
                               double *work)
{
    double *kb = work, *Yb = work + d;
    for (int64_t i = 0; i < d; ++i) kb[i] = hstep * lam[i];
    g(ctx, y, kb, Yb);
    for (int64_t i = 0; i < d; ++i) lam[i] += Yb[i];
}

/* Reverse of one step of tab_step's map: with the stages Y_s recomputed
   forward, the stage adjoints are, for s = n_stages down to 1,
     kb_s = h b_s lam + h a_{s+1} Yb_{s+1}  (the second term absent for the
            last stage),   Yb_s = J(Y_s)^T kb_s,
   and lam_n = lam + sum_s Yb_s; the vjp callback adds (df/dtheta)^T kb_s. */
static void tab_adjoint_step(const double *tab, int64_t d, double hstep, rhs_fn f, vjp_fn g, void *ctx,
                             const double *y, double *lam, double *work)
{
    const int ns = (int)tab[0];
    double *Ys = work, *k = work + 4 * d, *kb = work + 5 * d, *Yb = work + 6 * d, *Ysum = work + 7 * d;
    for (int64_t i = 0; i < d; ++i) Ys[i] = y[i];
    for (int st = 2; st <= ns; ++st) {
        f(ctx, Ys + (st - 2) * d, k);
        for (int64_t i = 0; i < d; ++i) Ys[(st - 1) * d + i] = y[i] + hstep * tab[st - 1] * k[i];
    }
    for (int64_t i = 0; i < d; ++i) Ysum[i] = 0.0;
    for (int st = ns; st >= 1; --st) {
        for (int64_t i = 0; i < d; ++i) {
            kb[i] = hstep * tab[3 + st] * lam[i];
            if (st < ns) kb[i] += hstep * tab[st] * Yb[i];
        }
        g(ctx, Ys + (st - 1) * d, kb, Yb);
        for (int64_t i = 0; i < d; ++i) Ysum[i] += Yb[i];
    }
    for (int64_t i = 0; i < d; ++i) lam[i] += Ysum[i];
}

static void adjoint_step(int order, const double *tab, int64_t d, double hstep, rhs_fn f, vjp_fn g, void *ctx,
                         const double *y, double *lam, double *work)
{
    if (order == 0) tab_adjoint_step(tab, d, hstep, f, g, ctx, y, lam, work);
    else if (order == 1) euler_adjoint_step(d, hstep, g, ctx, y, lam, work);
    else rk4_adjoint_step(d, hstep, f, g, ctx, y, lam, work);
}

static void lin_vjp(void *c, const double *y, const double *v, double *u)
{
    const lin_ctx *L = (const lin_ctx *)c;
    (void)y;
    for (int64_t j = 0; j < L->d; ++j) {
        double acc = 0.0;
        for (int64_t i = 0; i < L->d; ++i) acc += L->A[i * L->d + j] * v[i];
        u[j] = acc;
    }
}

/* Adjoint of nsteps RK4 (order 4), Euler (order 1) or tableau (order 0, tab) steps of dy/dt = A y:
   lam (adjoint of y at the end) is carried back to the adjoint of the
   initial state. */
int orc_linear_adjoint(int64_t d, const double *A, const double *y0, double h, int64_t nsteps, double *lam,
                       int order, const double *tab)
{
    double *traj = (double *)malloc(sizeof(double) * (size_t)d * (size_t)(nsteps + 1));
    double *work = (double *)malloc(sizeof(double) * 8 * (size_t)d);
    if (!traj || !work) { free(traj); free(work); return -1; }
    lin_ctx c = {d, A};
    memcpy(traj, y0, sizeof(double) * (size_t)d);
    for (int64_t k = 0; k < nsteps; ++k) {
        memcpy(traj + (k + 1) * d, traj + k * d, sizeof(double) * (size_t)d);
        take_step(order, tab, d, h, lin_rhs, &c, traj + (k + 1) * d, work);
    }
    for (int64_t k = nsteps - 1; k >= 0; --k)
        adjoint_step(order, tab, d, h, lin_rhs, lin_vjp, &c, traj + k * d, lam, work);
    free(traj);
    free(work);
    return 0;
}

typedef struct { const orc_net *net; const double *iext; orc_grads *g; } net_adj_ctx;

static void net_rhs_adj(void *c, const double *y, double *dy)
{
    const net_adj_ctx *nc = (const net_adj_ctx *)c;
    orc_rhs(nc->net, nc->iext, y, dy);
}

static void net_vjp(void *c, const double *y, const double *v, double *u)
{
    const net_adj_ctx *nc = (const net_adj_ctx *)c;
    orc_vjp(nc->net, nc->iext, y, v, u, nc->g);
}

/* Gradient of the linear functional L = sum_f sum_i dLdV[f][i] V_i(frame f)
   over the RK4 trajectory of nsteps steps from y0 (first step at global
   index step0; frame f is the state after global step k with
   k % rec_stride == 0, in order).  Outputs the adjoint of y0 (grad_y0[dim]),
   dL/dw (grad_w[S]) and dL/d(neuron-type parameters) (grad_np, row per
   type), for RK4 (order 4), Euler (order 1) or tableau (order 0, tab) steps.  Memory: states are
   kept every `ckpt` steps and each segment is recomputed.  Returns 0, or -1
   on allocation failure. */
int orc_adjoint(const orc_net *net, const double *y0, int64_t step0, int64_t nsteps, int64_t rec_stride,
                const double *dLdV, double *grad_y0, double *grad_w, double *grad_np, int64_t ckpt, int order,
                const double *tab)
{
    const int64_t d = 4 * net->N + 2 * net->S;
    if (ckpt < 1) ckpt = 1;
    const int64_t nck = (nsteps + ckpt - 1) / ckpt + 1;
    double *cks = (double *)malloc(sizeof(double) * (size_t)d * (size_t)nck);
    double *seg = (double *)malloc(sizeof(double) * (size_t)d * (size_t)(ckpt + 1));
    double *work = (double *)malloc(sizeof(double) * (8 * (size_t)d + 2 * (size_t)net->N));
    if (!cks || !seg || !work) { free(cks); free(seg); free(work); return -1; }
    double *iext = work + 8 * d;
    orc_grads g = {grad_w, grad_np};
    net_ctx fc = {net, iext};
    net_adj_ctx ac = {net, iext, &g};

    /* forward: checkpoints every ckpt steps */
    memcpy(cks, y0, sizeof(double) * (size_t)d);
    {
        double *y = seg;
        memcpy(y, y0, sizeof(double) * (size_t)d);
        for (int64_t k = 0; k < nsteps; ++k) {
            orc_input(net, step0 + k, iext);
            take_step(order, tab, d, net->dt, net_rhs, &fc, y, work);
            if ((k + 1) % ckpt == 0) memcpy(cks + ((k + 1) / ckpt) * d, y, sizeof(double) * (size_t)d);
        }
    }
    /* frames: global steps k in (step0, step0 + nsteps] with k % rec_stride == 0 */
    int64_t nframes = 0;
    if (rec_stride > 0)
        for (int64_t k = step0 + 1; k <= step0 + nsteps; ++k) nframes += (k % rec_stride) == 0;
    int64_t frame = nframes - 1;

    double *lam = grad_y0;
    for (int64_t i = 0; i < d; ++i) lam[i] = 0.0;
    /* the last state may itself be a frame */
    if (rec_stride > 0 && (step0 + nsteps) % rec_stride == 0 && frame >= 0) {
        for (int64_t i = 0; i < net->N; ++i) lam[i] += dLdV[frame * net->N + i];
        --frame;
    }
    for (int64_t c = (nsteps - 1) / ckpt; c >= 0; --c) {
        const int64_t k0 = c * ckpt, k1 = (k0 + ckpt < nsteps) ? k0 + ckpt : nsteps;
        /* recompute the segment's step states */
        memcpy(seg, cks + c * d, sizeof(double) * (size_t)d);
        for (int64_t k = k0; k < k1 - 1; ++k) {
            memcpy(seg + (k - k0 + 1) * d, seg + (k - k0) * d, sizeof(double) * (size_t)d);
            orc_input(net, step0 + k, iext);
            take_step(order, tab, d, net->dt, net_rhs, &fc, seg + (k - k0 + 1) * d, work);
        }
        for (int64_t k = k1 - 1; k >= k0; --k) {
            orc_input(net, step0 + k, iext);
            adjoint_step(order, tab, d, net->dt, net_rhs_adj, net_vjp, &ac, seg + (k - k0) * d, lam, work);
            /* state y_{step0+k} is a frame when its global index qualifies */
            if (rec_stride > 0 && k > 0 && (step0 + k) % rec_stride == 0 && frame >= 0) {
                for (int64_t i = 0; i < net->N; ++i) lam[i] += dLdV[frame * net->N + i];
                --frame;
            }
        }
    }
    free(cks);
    free(seg);
    free(work);
    return 0;
}
