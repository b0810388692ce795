"""Forward Euler (the paper's first-order method, Eq. euler) on the GPU against
the oracle's Euler step, in every execution path, and its bitwise
consistency between paths and launch forms."""
import numpy as np
import pytest

import oracle
from paper_1906_03958_gb300 import netgen as ng
from tests.helpers import grad_error
from tests.helpers import step_error

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-5


def _net(spec, **kw):
    from paper_1906_03958_gb300 import psst
    return psst.Network(spec, method=psst.METHOD_EULER, **kw)


def _euler_state(spec, n, step0):
    return oracle.integrate(spec, oracle.rest_state(spec), n, step0=step0, order=1)[0].astype(np.float32)


@pytest.mark.parametrize("case,gate_mode", [("al_cta", 0), ("al_cta", 1), ("al_cta_random_gates", 0),
                                            ("sparse_grid", 0), ("sparse_grid", 1), ("independent", 0)])
def test_euler_single_step_error(case, gate_mode):
    # per-pair and per-synapse gate layouts (gate_mode 1, or a state whose
    # pair gates differ), CTA and grid modes, independent neurons
    from paper_1906_03958_gb300 import psst
    if case.startswith("al_cta"):
        spec, mode, step0 = ng.antennal_lobe(seed=81), psst.MODE_CTA, 9980
    elif case == "sparse_grid":
        spec, mode, step0 = ng.sparse_large(seed=82, n_e=1600, n_i=400), psst.MODE_GRID, 300
    else:
        spec, mode, step0 = ng.independent(2000, seed=83, n_nets=2, rate_hz=200.0), psst.MODE_CTA, 1990
    N, S = spec.n_neurons, spec.n_synapses
    y32 = _euler_state(spec, 40, step0)
    if case == "al_cta_random_gates":
        rng = np.random.default_rng(7)
        y32[4 * N:4 * N + S] = rng.uniform(0.0, 1.0, S).astype(np.float32)
        y32[4 * N + S:] = rng.uniform(0.0, 1.0, S).astype(np.float32)
    y64, _ = oracle.integrate(spec, y32.astype(np.float64), 1, step0=step0 + 40, order=1)
    with _net(spec, init_state=y32, mode=mode, gate_mode=gate_mode) as net:
        if case == "al_cta_random_gates" or gate_mode == 1:
            assert net.info()["n_pair_gate_nets"] == 0
        net.set_step(step0 + 40)
        net.integrate(1)
        net.status()
        got = net.get_state_numpy()
    assert step_error(got, y64, N, S) <= STEP_TOL


@pytest.mark.parametrize("gate_mode", [0, 1])
def test_euler_cta_equals_grid_and_chunked_and_graph_bitwise(gate_mode):
    # odd and even step counts per call (the grid's final gate maps sit in the
    # table of the step count's parity)
    from paper_1906_03958_gb300 import psst
    spec = ng.antennal_lobe(seed=84)
    y0 = oracle.rest_state(spec).astype(np.float32)
    out = []
    for mode, chunks, graph in ((psst.MODE_CTA, [301], False), (psst.MODE_GRID, [301], False),
                                (psst.MODE_GRID, [100, 101, 100], False),
                                (psst.MODE_CTA, [100, 100, 101], False), (psst.MODE_CTA, [43] * 7, True)):
        with _net(spec, init_state=y0, mode=mode, item_chunks=2, rec_stride=5, rec_capacity=100,
                  gate_mode=gate_mode) as net:
            net.set_graph_mode(graph)
            net.set_step(9900)
            for c in chunks:
                net.integrate(c)
            net.status()
            out.append((net.get_state_numpy(), net.read_record()))
    for y, rec in out[1:]:
        np.testing.assert_array_equal(y, out[0][0])
        np.testing.assert_array_equal(rec, out[0][1])
    assert np.ptp(out[0][0][:spec.n_neurons]) > 10.0  # the pulse drives spikes


def test_euler_trajectory_tracks_oracle_euler():
    # 300 Euler steps of the 20-neuron network: FP32 against FP64 Euler
    spec = ng.plain20(seed=85)
    y0 = oracle.rest_state(spec)
    _, rec64 = oracle.integrate(spec, y0, 300, rec_stride=10, order=1)
    with _net(spec, init_state=y0.astype(np.float32), rec_stride=10, rec_capacity=30) as net:
        net.integrate(300)
        net.status()
        rec32 = net.read_record()
    assert np.max(np.abs(rec32 - rec64)) < 1e-2


GRAD_TOL = 1e-3


def _diff_spec(seed, sets=1):
    _, spec = ng.differentiated(n_sets=sets, seed=seed, n_pn=12, n_ln=4)
    spec.pulse_on[:] = 5
    spec.pulse_off[:] = 10_000
    return spec


def _euler_adjoint(spec, nsteps, dLdV, stride, ckpt=50, step0=0):
    import torch
    with _net(spec, rec_stride=stride, rec_capacity=nsteps // stride + 1) as net:
        net.set_step(step0)
        gw, gp, gy = net.adjoint(nsteps, torch.from_numpy(dLdV.astype(np.float32)).cuda(), ckpt)
        net.status()
        return gw.cpu().numpy(), gp.cpu().numpy(), gy.cpu().numpy()


@pytest.mark.parametrize("sets,ckpt", [(1, 100), (3, 64)])
def test_euler_adjoint_matches_oracle_euler_adjoint(sets, ckpt):
    # discrete adjoint of the Euler map (one stage, kb = h lam) against the
    # oracle's FP64 Euler adjoint, for one network and a batch of three
    spec = _diff_spec(seed=87 + sets, sets=sets)
    rng = np.random.default_rng(sets)
    nsteps, stride = 800, 8
    g = rng.standard_normal((nsteps // stride, spec.n_neurons))
    gy64, gw64, gp64 = oracle.adjoint(spec, oracle.rest_state(spec), nsteps, g, stride, ckpt=ckpt, order=1)
    gw, gp, gy = _euler_adjoint(spec, nsteps, g, stride, ckpt=ckpt)
    for b in range(spec.n_nets):
        s0, s1 = spec.row_ptr[spec.net_neuron_off[b]], spec.row_ptr[spec.net_neuron_off[b + 1]]
        assert grad_error(gw[s0:s1], gw64[s0:s1]) <= GRAD_TOL
        assert grad_error(gp[2 * b:2 * b + 2], gp64[2 * b:2 * b + 2]) <= GRAD_TOL
    N = spec.n_neurons
    assert grad_error(gy.ravel(), gy64[:4 * N]) <= GRAD_TOL
    # not the RK4 adjoint: the two maps' gradients differ by more than the bar
    _, gw_rk4, _ = oracle.adjoint(spec, oracle.rest_state(spec), nsteps, g, stride, ckpt=ckpt, order=4)
    assert grad_error(gw_rk4, gw64) > 10 * GRAD_TOL


def test_euler_adjoint_vs_fp64_finite_differences():
    # weights and conductances, central differences with h = 1e-6 max(1, |theta|)
    # on the FP64 Euler map; the differences' own rounding noise,
    # 4 eps sum|terms of L| / h, is admitted on top of the bar
    spec = _diff_spec(seed=90)
    net = oracle.OracleNet(spec)
    rng = np.random.default_rng(5)
    nsteps, stride = 500, 5
    g = rng.standard_normal((nsteps // stride, spec.n_neurons))
    y0 = oracle.rest_state(net)
    gw, gp, _ = _euler_adjoint(spec, nsteps, g, stride)

    def loss():
        _, rec = oracle.integrate(net, y0, nsteps, rec_stride=stride, order=1)
        return float(np.sum(rec * g))

    def fd(arr, idx):
        x0 = arr[idx]
        h = 1e-6 * max(1.0, abs(x0))
        arr[idx] = x0 + h
        lp = loss()
        arr[idx] = x0 - h
        lm = loss()
        arr[idx] = x0
        return (lp - lm) / (2 * h)

    _, rec = oracle.integrate(net, y0, nsteps, rec_stride=stride, order=1)
    fd_noise = 4.0 * np.finfo(float).eps * float(np.sum(np.abs(rec * g))) / 1e-6
    nz = np.nonzero(net.w)[0]
    coords = [("w", int(k)) for k in rng.choice(nz, 4, replace=False)] + \
             [("w", int(k)) for k in rng.choice(np.nonzero(net.w == 0)[0], 2, replace=False)]
    P = net.nparams.reshape(-1, 9)
    coords += [("p", (0, 1)), ("p", (0, 2)), ("p", (1, 3)), ("p", (1, 7))]
    scale_w = np.abs(gw).max()
    for kind, idx in coords:
        if kind == "w":
            want, got, scale = fd(net.w, idx), gw[idx], scale_w
        else:
            want, got, scale = fd(P, idx), gp[idx], abs(fd(P, idx))
        assert abs(got - want) <= GRAD_TOL * max(abs(want), 1e-2 * scale) + fd_noise, (kind, idx, got, want)


def test_euler_adjoint_checkpoint_spacing_step_offset_and_recorded_span():
    import torch
    spec = _diff_spec(seed=91, sets=2)
    rng = np.random.default_rng(6)
    nsteps, stride, step0 = 240, 4, 2
    frames = (step0 + nsteps) // stride - step0 // stride
    g = rng.standard_normal((frames, spec.n_neurons))
    a = _euler_adjoint(spec, nsteps, g, stride, ckpt=7, step0=step0)
    b = _euler_adjoint(spec, nsteps, g, stride, ckpt=240, step0=step0)
    for x, y in zip(a, b):
        assert grad_error(x, y) <= 1e-5
    _, gw64, _ = oracle.adjoint(spec, oracle.rest_state(spec), nsteps, g, stride, step0=step0, order=1)
    assert grad_error(a[0], gw64) <= GRAD_TOL
    # the span of an Euler integrate call whose checkpoints were recorded
    gt = torch.from_numpy(g.astype(np.float32)).cuda()
    with _net(spec, rec_stride=stride, rec_capacity=frames) as net:
        net.set_step(step0)
        net.record_checkpoints(60, nsteps)
        net.integrate(nsteps)
        rec = net.adjoint(nsteps, gt, 0)
        net.status()
        assert grad_error(rec[0].cpu().numpy(), a[0]) <= 1e-5
        assert grad_error(rec[1].cpu().numpy(), a[1]) <= 1e-5
