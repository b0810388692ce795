"""Pins of the oracle's discrete RK4 adjoint (CPU only).

* the Jacobian-transpose product of the right-hand side against central
  finite differences of the (separately pinned) right-hand side;
* the reverse RK4 driver against the closed form on y' = A y:
  lam_0 = (P4(hA)^T)^n lam_T with P4 the degree-4 Taylor polynomial;
* whole-trajectory gradients (initial state, weights, neuron-type
  parameters) against FP64 central finite differences of the forward map;
* independence of the checkpoint spacing.
"""
import numpy as np
import pytest

import oracle
from paper_1906_03958_gb300 import netgen as ng


def _small_al(seed=3):
    spec = ng.antennal_lobe(seed=seed, n_pn=6, n_ln=3, p=0.6, w_max=(0.3, 0.6, 0.3), odor_amp=30.0)
    spec.pulse_on[:] = 0
    spec.pulse_off[:] = 10_000
    return spec


def _random_state(spec, rng):
    net = oracle.OracleNet(spec)
    N, S = net.N, net.S
    y = np.empty(net.dim)
    y[:N] = rng.uniform(-80, 40, N)
    y[N:4 * N] = rng.uniform(0.05, 0.95, 3 * N)
    y[4 * N:4 * N + S] = rng.uniform(0.05, 0.95, S)
    y[4 * N + S:] = rng.uniform(0.1, 5.0, S)
    return y


def test_vjp_equals_fd_jacobian_transpose():
    spec = _small_al()
    net = oracle.OracleNet(spec)
    rng = np.random.default_rng(1)
    y = _random_state(spec, rng)
    v = rng.standard_normal(net.dim)
    u, gw, gnp = oracle.vjp(net, y, v, step=5)
    # J^T v column by column: (d f / d y_c) . v by central differences
    fd = np.empty(net.dim)
    for c in range(net.dim):
        h = 1e-6 * max(1.0, abs(y[c]))
        yp, ym = y.copy(), y.copy()
        yp[c] += h
        ym[c] -= h
        fd[c] = (oracle.rhs(net, yp, 5) - oracle.rhs(net, ym, 5)) @ v / (2 * h)
    np.testing.assert_allclose(u, fd, rtol=1e-6, atol=1e-6 * np.abs(fd).max())
    # weights
    for k in rng.choice(net.S, 8, replace=False):
        w0 = net.w[k]
        h = 1e-6 * max(1.0, abs(w0))
        net.w[k] = w0 + h
        fp = oracle.rhs(net, y, 5) @ v
        net.w[k] = w0 - h
        fm = oracle.rhs(net, y, 5) @ v
        net.w[k] = w0
        assert gw[k] == pytest.approx((fp - fm) / (2 * h), rel=1e-6, abs=1e-9)
    # every neuron-type parameter
    P = net.nparams.reshape(-1, 9)
    for t in range(P.shape[0]):
        for c in range(9):
            p0 = P[t, c]
            h = 1e-6 * max(1.0, abs(p0))
            P[t, c] = p0 + h
            fp = oracle.rhs(net, y, 5) @ v
            P[t, c] = p0 - h
            fm = oracle.rhs(net, y, 5) @ v
            P[t, c] = p0
            assert gnp[t, c] == pytest.approx((fp - fm) / (2 * h), rel=1e-6, abs=1e-9), (t, c)


@pytest.mark.parametrize("order", [4, 1])
def test_linear_adjoint_closed_form(order):
    # one step maps y to P(hA) y with P the degree-`order` Taylor polynomial
    # (RK4: 4, Euler: 1), so the adjoint carries lam back by (P^T)^n
    A = np.array([[-1.0, 4.0, 0.0], [0.0, -1.0, 4.0], [0.5, 0.0, -2.0]])
    y0 = np.array([1.0, 2.0, -1.0])
    h, n = 0.05, 40
    lam_T = np.array([0.3, -1.2, 0.7])
    hA = h * A
    P, term = np.eye(3), np.eye(3)
    for k in range(1, order + 1):
        term = term @ hA / k
        P = P + term
    want = np.linalg.matrix_power(P.T, n) @ lam_T
    np.testing.assert_allclose(oracle.linear_adjoint(A, y0, h, n, lam_T, order=order), want, rtol=1e-13,
                               atol=1e-13)


def _loss(net, y0, nsteps, g, stride, step0=0, order=4, tableau=None):
    _, rec = oracle.integrate(net, y0, nsteps, step0=step0, rec_stride=stride, order=order, tableau=tableau)
    return float(np.sum(rec * g))


# Heun's third-order method: a_21 = 1/3, a_32 = 2/3, b = (1/4, 0, 3/4);
# the midpoint method (first weight zero): a_21 = 1/2, b = (0, 1)
HEUN3 = ([1.0 / 3.0, 2.0 / 3.0], [0.25, 0.0, 0.75])
MIDPOINT = ([0.5], [0.0, 1.0])


@pytest.mark.parametrize("order,tableau", [(4, None), (1, None), (0, HEUN3), (0, MIDPOINT)])
def test_trajectory_gradient_vs_fd(order, tableau):
    spec = _small_al(seed=4)
    net = oracle.OracleNet(spec)
    rng = np.random.default_rng(2)
    y0 = oracle.rest_state(net)
    y0[: net.N] += rng.uniform(-5, 15, net.N)
    nsteps, stride, step0 = 400, 10, 3
    frames = sum(1 for k in range(step0 + 1, step0 + nsteps + 1) if k % stride == 0)
    g = rng.standard_normal((frames, net.N))
    gy, gw, gnp = oracle.adjoint(net, y0, nsteps, g, stride, step0=step0, ckpt=37, order=order, tableau=tableau)

    def fd(setter, x0):
        h = 1e-6 * max(1.0, abs(x0))
        setter(x0 + h)
        lp = _loss(net, y0, nsteps, g, stride, step0, order, tableau)
        setter(x0 - h)
        lm = _loss(net, y0, nsteps, g, stride, step0, order, tableau)
        setter(x0)
        return (lp - lm) / (2 * h)

    scale = np.abs(gw).max()
    # central differences with step h carry a rounding error of about
    # eps * sum|terms of L| / h (h = 1e-6 relative: ~1e-6 absolute here),
    # which the bound for the smallest weight gradients must admit
    _, rec = oracle.integrate(net, y0, nsteps, step0=step0, rec_stride=stride, order=order, tableau=tableau)
    fd_noise = 4.0 * np.finfo(float).eps * float(np.sum(np.abs(rec * g))) / 1e-6
    for k in rng.choice(net.S, 10, replace=False):
        want = fd(lambda x: net.w.__setitem__(k, x), net.w[k])
        assert abs(gw[k] - want) <= 1e-6 * max(abs(want), 1e-3 * scale) + fd_noise, (k, gw[k], want)
    P = net.nparams.reshape(-1, 9)
    for t, c in [(0, 1), (0, 2), (1, 3), (1, 7), (0, 0), (1, 6)]:
        want = fd(lambda x: P.__setitem__((t, c), x), P[t, c])
        assert gnp[t, c] == pytest.approx(want, rel=1e-6), (t, c)
    ys = y0.copy()
    for c in [0, net.N + 2, 2 * net.N + 1, 4 * net.N + 3, 4 * net.N + net.S + 5]:
        def setter(x, c=c):
            y0[c] = x
        want = fd(setter, y0[c])
        assert gy[c] == pytest.approx(want, rel=1e-6, abs=1e-9 * np.abs(gy).max()), c
    np.testing.assert_array_equal(y0, ys)


def test_checkpoint_spacing_does_not_change_gradients():
    spec = _small_al(seed=5)
    net = oracle.OracleNet(spec)
    rng = np.random.default_rng(3)
    y0 = oracle.rest_state(net)
    g = rng.standard_normal((30, net.N))
    out = [oracle.adjoint(net, y0, 300, g, 10, ckpt=c) for c in (1, 13, 300)]
    for o in out[1:]:
        for a, b in zip(out[0], o):
            np.testing.assert_allclose(a, b, rtol=1e-12, atol=1e-14)


def test_full_size_differentiated_adjoint_matches_finite_differences():
    # The stored FP64 oracle adjoint of the full differentiated workload
    # (120 neurons, dense weights + GABA_B, 20,000 RK4 steps, checkpoints
    # every 1,000; mean-square PN trace loss; tests/golden/make_adjoint_al120.py)
    # against the stored
    # FP64 central differences on 10 coordinates, each taken at the step of
    # the ladder whose neighbour agrees best, within 1e-4 of the difference
    # plus its own error bound.
    import os
    from tests.helpers import fd_reference
    G = np.load(os.path.join(os.path.dirname(__file__), "golden", "adjoint_al120_20k.npz"))
    ref, err = fd_reference(G["fd"])
    got = [G["gw"][k] for k in G["fd_w_index"]] + [G["gp"][tuple(p)] for p in G["fd_p_index"]]
    for c, (x, want, e) in enumerate(zip(got, ref, err)):
        assert abs(x - want) <= 1e-4 * abs(want) + e, (c, x, want, e)
    # the loss the gradients belong to is the one the script describes
    from tests.golden import make_adjoint_al120 as gold
    assert int(G["nsteps"]) == gold.NSTEPS and int(G["n_pn"]) == gold.N_PN
