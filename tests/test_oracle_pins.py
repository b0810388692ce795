"""Pins of the FP64 oracle to facts outside itself.

Each test checks the oracle against a closed form, a textbook fact, an
invariant or a library routine, chosen so that a dropped term, a wrong sign,
a wrong index or a swapped operand in ``oracle/psst_oracle.c`` fails one of
them.  No GPU is needed.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate as sint
from scipy import linalg

import oracle
from paper_1906_03958_gb300 import netgen as ng

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hh_textbook.json")))

PASSIVE = dict(C=1.0, gNa=0.0, gK=0.0, gL=0.0, ENa=50.0, EK=-77.0, EL=-54.387,
               gKL=0.0, EKL=-95.0)


# ----------------------------------------------------------- RK4 / Euler map

def _A2():
    return np.array([[-0.3, 2.0], [-2.0, -0.3]])


def _A3():
    return np.array([[-1.0, 4.0, 0.0], [0.0, -1.0, 4.0], [0.5, 0.0, -2.0]])


@pytest.mark.parametrize("A", [_A2(), _A3()])
def test_rk4_one_step_is_degree4_taylor_polynomial(A):
    # Sec. "Brain simulations ...", RK4 paragraph: for y' = A y one classic
    # RK4 step is exactly sum_{k<=4} (hA)^k / k! applied to y0.
    h = 0.1
    y0 = np.arange(1.0, A.shape[0] + 1.0)
    hA = h * A
    P = np.eye(len(y0))
    term = np.eye(len(y0))
    for k in range(1, 5):
        term = term @ hA / k
        P = P + term
    got = oracle.linear_integrate(A, y0, h, 1, order=4)
    np.testing.assert_allclose(got, P @ y0, rtol=1e-14, atol=1e-14)
    # forward Euler, Eq. (euler): I + hA
    got1 = oracle.linear_integrate(A, y0, h, 1, order=1)
    np.testing.assert_allclose(got1, (np.eye(len(y0)) + hA) @ y0, rtol=1e-15, atol=1e-15)


@pytest.mark.parametrize("order,slope,h0", [(4, 4.0, 0.1), (1, 1.0, 0.005)])
def test_global_convergence_order(order, slope, h0):
    # local error O(dt^5) for RK4 -> global O(dt^4); Euler global O(dt)
    A = _A2()
    y0 = np.array([1.0, -0.5])
    T = 2.0
    exact = linalg.expm(A * T) @ y0
    errs = []
    hs = [h0, h0 / 2, h0 / 4, h0 / 8]
    for h in hs:
        y = oracle.linear_integrate(A, y0, h, int(round(T / h)), order=order)
        errs.append(np.max(np.abs(y - exact)))
    slopes = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert all(abs(s - slope) < 0.1 for s in slopes), slopes


# ------------------------------------------------------------ HH functions

def test_rate_function_special_points():
    lim = GOLDEN["rate_limits"]
    assert oracle.rates(-40.0)[0] == lim["alpha_m_at_minus40"]
    assert oracle.rates(-55.0)[4] == lim["alpha_n_at_minus55"]
    # continuity through the removable singularities
    for dv in (1e-9, -1e-9, 1e-5, -1e-5):
        assert abs(oracle.rates(-40.0 + dv)[0] - (1.0 + dv / 20.0)) < 1e-9
        assert abs(oracle.rates(-55.0 + dv)[4] - (0.1 + dv / 200.0)) < 1e-10
    # prefactors where each exponent vanishes
    r65 = oracle.rates(-65.0)
    assert r65[1] == pytest.approx(4.0, rel=1e-15)      # beta_m
    assert r65[2] == pytest.approx(0.07, rel=1e-15)     # alpha_h
    assert r65[5] == pytest.approx(0.125, rel=1e-15)    # beta_n
    assert oracle.rates(-35.0)[3] == pytest.approx(0.5, rel=1e-15)  # beta_h midpoint
    # e-fold voltages (18, 20, 80 mV) and the beta_h slope (10 mV)
    assert oracle.rates(-83.0)[1] / r65[1] == pytest.approx(math.e, rel=1e-13)
    assert oracle.rates(-85.0)[2] / r65[2] == pytest.approx(math.e, rel=1e-13)
    assert oracle.rates(-145.0)[5] / r65[5] == pytest.approx(math.e, rel=1e-13)
    assert oracle.rates(-25.0)[3] == pytest.approx(1.0 / (1.0 + math.exp(-1.0)), rel=1e-14)
    # linear asymptotes far above the singular points: 0.1 (V+40), 0.01 (V+55)
    assert oracle.rates(160.0)[0] == pytest.approx(20.0, rel=1e-8)
    assert oracle.rates(245.0)[4] == pytest.approx(3.0, rel=1e-8)
    # and exponentially small far below
    assert oracle.rates(-240.0)[0] < 1e-6 and oracle.rates(-255.0)[4] < 1e-7


def test_rest_gates_match_textbook():
    g = GOLDEN["rest_gates"]
    m, h, n = oracle.steady_gates(g["V_mV"])
    assert abs(m - g["m_inf"]) < g["abs_tol"]
    assert abs(h - g["h_inf"]) < g["abs_tol"]
    assert abs(n - g["n_inf"]) < g["abs_tol"]


def test_rest_current_balance():
    spec = ng.single_network([0], [0.0], [], [], [], [], ng.neuron_table(ng.HH),
                             ng.synapse_table(ng.ACH))
    y = oracle.rest_state(spec)
    dy = oracle.rhs(spec, y)
    assert abs(dy[0]) < GOLDEN["rest_current_balance"]["max_abs_ionic_current_uA_cm2"]
    assert np.all(np.abs(dy[1:4]) < 1e-15)  # gates exactly at their steady state


def _single(I):
    return ng.single_network([0], [I], [], [], [], [], ng.neuron_table(ng.HH),
                             ng.synapse_table(ng.ACH))


def test_repetitive_firing_regimes():
    rf = GOLDEN["repetitive_firing"]
    spec = _single(rf["no_sustained_firing_at_uA_cm2"])
    _, rec = oracle.integrate(spec, oracle.rest_state(spec), 20000, rec_stride=1)
    st = oracle.spike_times(rec, 0.01)[0]
    assert len(st[st > 50.0]) == 0 and len(st) <= 1
    spec = _single(rf["sustained_firing_at_uA_cm2"])
    _, rec = oracle.integrate(spec, oracle.rest_state(spec), 20000, rec_stride=1)
    st = oracle.spike_times(rec, 0.01)[0]
    isi = np.diff(st)
    lo, hi = rf["isi_ms_range_at_10"]
    assert len(st) >= 12
    assert lo < np.median(isi[2:]) < hi
    assert rec.max() > 30.0  # overshoot of the action potential


def test_gates_stay_in_unit_interval():
    spec = ng.plain20(weight_scale=0.1)
    y = oracle.rest_state(spec)
    net = oracle.OracleNet(spec)
    N, S = net.N, net.S
    for chunk in range(40):
        y, _ = oracle.integrate(net, y, 250, step0=250 * chunk)
        gates = y[N:4 * N]
        assert gates.min() >= 0.0 and gates.max() <= 1.0
        assert y[4 * N:4 * N + S].min() >= 0.0 and y[4 * N:4 * N + S].max() <= 1.0


def test_transmitter_midpoint_and_limits():
    for Vp, Kp in ((2.0, 5.0), (-20.0, 2.0)):
        assert oracle.transmitter(Vp, Vp, Kp) == 0.5
        assert oracle.transmitter(Vp + Kp, Vp, Kp) == pytest.approx(1 / (1 + math.exp(-1)), rel=1e-15)
        assert oracle.transmitter(Vp + 100 * Kp, Vp, Kp) == pytest.approx(1.0, abs=1e-15)


# ------------------------------------------------------------ synapses

def _passive_net(V0s, post, pre, w, stype, stab):
    n = len(V0s)
    spec = ng.single_network(np.zeros(n), np.zeros(n), post, pre, w, stype,
                             ng.neuron_table(PASSIVE), stab)
    y = oracle.rest_state(spec)
    y[:n] = V0s
    return spec, y


def _f32(q):
    """The parameters as the network actually holds them (float32)."""
    return {k: float(np.float32(v)) for k, v in q.items()}


DT32 = float(np.float32(0.01))


def _T(V, q):
    return 1.0 / (1.0 + math.exp(-(V - q["Vp"]) / q["Kp"]))


def test_first_order_synapses_closed_form():
    # Passive neurons (no conductances, no input): presynaptic V stays at V0
    # exactly, so each gate relaxes as r(t) = r_inf (1 - exp(-k t)) with
    # k = a T + b, r_inf = a T / k; the postsynaptic neuron then obeys
    # V' = -sum_j w_j r_j(t) (V - E), with E = 0 for both synapses here:
    # V(t) = V0 exp(-sum_j w_j int_0^t r_j).
    q = _f32(ng.ACH)
    V0 = [10.0, -20.0, -50.0]
    w = [float(np.float32(0.3)), float(np.float32(0.2))]
    spec, y0 = _passive_net(V0, [2, 2], [0, 1], w, [0, 0], ng.synapse_table(q))
    t = 500 * DT32
    y, _ = oracle.integrate(spec, y0, 500)
    integ = 0.0
    for j, wj in enumerate(w):
        aT = q["a"] * _T(V0[j], q)
        k = aT + q["b"]
        rinf = aT / k
        r_t = rinf * (1 - math.exp(-k * t))
        assert y[12 + j] == pytest.approx(r_t, rel=1e-9)  # r of synapse j (post-sorted by pre)
        integ += wj * rinf * (t - (1 - math.exp(-k * t)) / k)
    assert y[2] == pytest.approx(V0[2] * math.exp(-integ), rel=1e-9)
    assert y[0] == V0[0] and y[1] == V0[1]


def test_mixed_reversal_potentials_vs_quadrature():
    # One excitatory (E = 0) and one inhibitory (E = -80) synapse onto a
    # passive neuron: V' = -(g_e(t) V + g_i(t) (V + 80)), solved here by
    # scipy's DOP853 with the closed-form conductances.
    qa, qb = _f32(ng.ACH), _f32(ng.GABA_A)
    V0 = [15.0, -5.0, -30.0]
    w = [float(np.float32(0.4)), 0.25]
    spec, y0 = _passive_net(V0, [2, 2], [0, 1], w, [0, 1], ng.synapse_table(qa, qb))
    t_end = 800 * DT32
    y, _ = oracle.integrate(spec, y0, 800)

    def g(t, j, q):
        aT = q["a"] * _T(V0[j], q)
        k = aT + q["b"]
        return w[j] * aT / k * (1 - math.exp(-k * t))

    sol = sint.solve_ivp(lambda t, v: [-(g(t, 0, qa) * (v[0] - qa["E"]) + g(t, 1, qb) * (v[0] - qb["E"]))],
                         (0, t_end), [V0[2]], method="DOP853", rtol=1e-12, atol=1e-12)
    assert y[2] == pytest.approx(sol.y[0, -1], rel=1e-8)


def test_second_order_gaba_b_closed_form():
    # Slow GABA_B pair with constant presynaptic V: r as above, and
    # s(t) = K3 r_inf [(1 - e^{-K4 t})/K4 - (e^{-k t} - e^{-K4 t})/(K4 - k)]
    # from s' = K3 r - K4 s, s(0) = 0; the postsynaptic V then follows
    # V - E = (V0 - E) exp(-w int_0^t s^4/(s^4+Kd)).
    q = _f32(ng.GABA_B)
    V0 = [20.0, -60.0]
    w = float(np.float32(0.003))  # small enough that V is still far from E at the end
    spec, y0 = _passive_net(V0, [1], [0], [w], [0], ng.synapse_table(q))
    nsteps = 20000
    t = nsteps * DT32
    y, _ = oracle.integrate(spec, y0, nsteps)
    aT = q["a"] * _T(V0[0], q)
    k = aT + q["b"]
    rinf = aT / k
    K3, K4, Kd, E = q["K3"], q["K4"], q["Kd"], q["E"]

    def r_of(t):
        return rinf * (1 - math.exp(-k * t))

    def s_of(t):
        return K3 * rinf * ((1 - math.exp(-K4 * t)) / K4 - (math.exp(-k * t) - math.exp(-K4 * t)) / (K4 - k))

    N, S = 2, 1
    assert y[4 * N] == pytest.approx(r_of(t), rel=1e-9)
    assert y[4 * N + S] == pytest.approx(s_of(t), rel=1e-9)
    G_int, _ = sint.quad(lambda u: s_of(u) ** 4 / (s_of(u) ** 4 + Kd), 0, t, limit=400,
                         epsabs=1e-13, epsrel=1e-13)
    assert y[1] == pytest.approx(E + (V0[1] - E) * math.exp(-w * G_int), rel=1e-8)


@pytest.mark.parametrize("cond", ["gL", "gKL"])
def test_single_leak_conductance_closed_form(cond):
    # one passive conductance g to reversal E_x: V(t) = E_x + (V0 - E_x) e^{-g t / C}
    erev = {"gL": "EL", "gKL": "EKL"}[cond]
    prm = _f32(dict(PASSIVE, C=1.5, **{cond: 0.2}))
    spec = ng.single_network([0], [0.0], [], [], [], [], ng.neuron_table(prm),
                             ng.synapse_table(ng.ACH))
    y0 = oracle.rest_state(spec, V0=-20.0)
    y, _ = oracle.integrate(spec, y0, 1000)
    t = 1000 * DT32
    E = prm[erev]
    assert y[0] == pytest.approx(E + (-20.0 - E) * math.exp(-prm[cond] * t / prm["C"]), rel=1e-10)


# ------------------------------------------------------------ inputs

def test_pulse_window_on_step_boundaries():
    # passive neuron: dV/dt = I/C is constant within a step, so RK4 is exact
    spec = ng.single_network([0], [0.5], [], [], [], [], ng.neuron_table(dict(PASSIVE, C=2.0)),
                             ng.synapse_table(ng.ACH), pulse_amp=[3.0], pulse_on=7, pulse_off=19)
    y0 = oracle.rest_state(spec)
    y, rec = oracle.integrate(spec, y0, 30, rec_stride=1)
    dt = np.float64(np.float32(0.01))
    drift = np.arange(1, 31) * 0.5 * dt / 2.0
    pulse = np.clip(np.arange(1, 31) - 7, 0, 12) * 3.0 * dt / 2.0
    np.testing.assert_allclose(rec[:, 0], -65.0 + drift + pulse, rtol=0, atol=1e-12)


def test_shot_noise_wiring():
    thresh = int(0.3 * (1 << 24))
    spec = ng.single_network([0, 0], [0.0, 0.0], [], [], [], [], ng.neuron_table(PASSIVE),
                             ng.synapse_table(ng.ACH), noise_seed=77, noise_thresh=thresh,
                             noise_amp=2.0)
    y0 = oracle.rest_state(spec)
    y, _ = oracle.integrate(spec, y0, 400, step0=1000)
    dt = np.float64(np.float32(0.01))
    for i in range(2):
        cnt = sum(oracle.noise_event(77, thresh, k, i) for k in range(1000, 1400))
        assert 80 < cnt < 160
        assert y[i] == pytest.approx(-65.0 + 2.0 * dt * cnt, abs=1e-11)


PHILOX_KAT = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "philox_kat.json")))


@pytest.mark.parametrize("vec", PHILOX_KAT["vectors"])
def test_philox_known_answer_vectors(vec):
    # The generator's published known-answer vectors (Salmon et al., SC'11;
    # tests/golden/philox_kat.json): all four output words, bit for bit.
    ctr = tuple(int(x, 16) for x in vec["ctr"])
    key = tuple(int(x, 16) for x in vec["key"])
    want = [int(x, 16) for x in vec["out"]]
    got = [int(x) for x in oracle.philox(ctr, key)]
    assert got == want, ["%08x" % g for g in got]


_TRITON_PHILOX = r"""
import os, sys, json
os.environ["TRITON_INTERPRET"] = "1"
import numpy as np, torch, triton, triton.language as tl

@triton.jit
def draw(out, c0p, c1p, c2p, c3p, seed, B: tl.constexpr):
    o = tl.arange(0, B)
    a, b, c, d = tl.philox(seed, tl.load(c0p + o), tl.load(c1p + o), tl.load(c2p + o), tl.load(c3p + o))
    tl.store(out + 4 * o, a)
    tl.store(out + 4 * o + 1, b)
    tl.store(out + 4 * o + 2, c)
    tl.store(out + 4 * o + 3, d)

ctr = np.array(json.loads(sys.argv[1]), dtype=np.uint32)
B = ctr.shape[0]
out = torch.zeros(4 * B, dtype=torch.int32)
cols = [torch.from_numpy(np.ascontiguousarray(ctr[:, j]).view(np.int32)) for j in range(4)]
draw[(1,)](out, *cols, int(sys.argv[2]), B=B)
print(json.dumps(out.numpy().view(np.uint32).reshape(B, 4).tolist()))
"""


def test_philox_matches_library_generator():
    # A second, independent implementation of the same generator: Triton's
    # tl.philox (Philox4x32 with 10 rounds, key = the 64-bit seed split into
    # low and high words), run by Triton's CPU interpreter in a child
    # process.  Random counters and a fixed key; all four words must agree.
    pytest.importorskip("triton")
    import subprocess
    import sys
    rng = np.random.default_rng(123)
    ctr = rng.integers(0, 1 << 32, size=(16, 4), dtype=np.uint64)
    seed = 0x0BADF00D1234ABCD
    r = subprocess.run([sys.executable, "-c", _TRITON_PHILOX, json.dumps(ctr.tolist()), str(seed)],
                       capture_output=True, text=True, timeout=600)
    if r.returncode != 0:
        pytest.skip("Triton's CPU interpreter is unavailable: " + r.stderr.strip().splitlines()[-1][:200])
    lib = np.array(json.loads(r.stdout.strip().splitlines()[-1]), dtype=np.uint64)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    for row, want in zip(ctr, lib):
        got = oracle.philox(tuple(int(x) for x in row), key)
        assert [int(x) for x in got] == [int(x) for x in want]


def test_philox_statistics():
    # Statistical properties, beside the exact pins above.
    words = []
    key = (0x1234ABCD, 0x0BADF00D)
    for c in range(1 << 14):
        words.extend(oracle.philox((c, 0, 7, 0), key))
    x = np.array(words, dtype=np.uint64)
    u = (x >> np.uint64(8)).astype(np.float64) / (1 << 24)
    assert abs(u.mean() - 0.5) < 3e-3
    assert abs(u.var() - 1 / 12) < 2e-3
    counts = np.bincount((u * 64).astype(int), minlength=64)
    chi2 = ((counts - len(u) / 64) ** 2 / (len(u) / 64)).sum()
    assert chi2 < 120  # 63 dof; p ~ 1e-5 tail
    bits = np.unpackbits(x.astype("<u4").view(np.uint8)).reshape(-1, 32).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 0.02)
    # avalanche: one flipped counter bit changes about half the output bits
    base = oracle.philox((5, 6, 7, 8), key)
    flips = []
    for b in range(32):
        o = oracle.philox((5 ^ (1 << b), 6, 7, 8), key)
        flips.append(sum(bin(int(a) ^ int(c)).count("1") for a, c in zip(base, o)))
    assert 56 < np.mean(flips) < 72
    # distinct keys give distinct streams
    assert not np.array_equal(oracle.philox((1, 2, 3, 4), (1, 0)), oracle.philox((1, 2, 3, 4), (2, 0)))


# ------------------------------------------------------- network invariants

def test_zero_weights_decouple_into_single_neurons():
    # the vectorised network with all weights 0 is N independent HH neurons
    spec = ng.plain20()
    spec.weight = np.zeros_like(spec.weight)
    y0 = oracle.rest_state(spec)
    y, rec = oracle.integrate(spec, y0, 2000, rec_stride=10)
    for i in (0, 7, 19):
        s1 = _single(float(spec.i_const[i]))
        y1, rec1 = oracle.integrate(s1, oracle.rest_state(s1), 2000, rec_stride=10)
        np.testing.assert_array_equal(rec[:, i], rec1[:, 0])


def test_batch_equals_separate_networks():
    a, b = ng.plain20(seed=11), ng.plain20(seed=12)
    both = ng.concat_specs([a, b])
    ya0, yb0 = oracle.rest_state(a), oracle.rest_state(b)
    yab, recab = oracle.integrate(both, oracle.rest_state(both), 500, rec_stride=5)
    ya, reca = oracle.integrate(a, ya0, 500, rec_stride=5)
    yb, recb = oracle.integrate(b, yb0, 500, rec_stride=5)
    np.testing.assert_array_equal(recab[:, :20], reca)
    np.testing.assert_array_equal(recab[:, 20:], recb)


def test_row_order_does_not_matter():
    # vectorisation/reordering of the synaptic sum changes results only by
    # rounding (the sum is over an unordered set of synapses)
    spec = ng.plain20(weight_scale=0.2)
    rng = np.random.default_rng(3)
    perm_spec = ng.NetworkSpec(**{k: getattr(spec, k) for k in spec.__dataclass_fields__})
    perm = np.arange(spec.n_synapses)
    for i in range(spec.n_neurons):
        lo, hi = spec.row_ptr[i], spec.row_ptr[i + 1]
        perm[lo:hi] = lo + rng.permutation(hi - lo)
    for k in ("pre", "weight", "syn_type"):
        setattr(perm_spec, k, getattr(spec, k)[perm])
    y0 = oracle.rest_state(spec)
    _, r1 = oracle.integrate(spec, y0, 1000, rec_stride=10)
    _, r2 = oracle.integrate(perm_spec, y0, 1000, rec_stride=10)
    np.testing.assert_allclose(r1, r2, rtol=0, atol=1e-9)
