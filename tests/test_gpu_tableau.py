"""Explicit Runge-Kutta maps of a given tableau (METHOD_TABLEAU: stage s
starts at y + dt a_s k_{s-1}) on the GPU: the classic and the one-stage
tableaus against the RK4 and Euler kernels bit for bit, other tableaus
against the oracle's map of the same tableau, bitwise consistency between
execution paths, and the discrete adjoint."""
import numpy as np
import pytest

import oracle
from paper_1906_03958_gb300 import netgen as ng
from tests.helpers import grad_error
from tests.helpers import step_error

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-5
GRAD_TOL = 1e-3
RK4 = ([0.5, 0.5, 1.0], [1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0])
EULER = ([], [1.0])
MIDPOINT = ([0.5], [0.0, 1.0])
RALSTON2 = ([2.0 / 3.0], [0.25, 0.75])
HEUN3 = ([1.0 / 3.0, 2.0 / 3.0], [0.25, 0.0, 0.75])


def _case(case):
    from paper_1906_03958_gb300 import psst
    if case in ("al_pair", "al_syn"):
        return ng.antennal_lobe(seed=96), psst.MODE_CTA, int(case == "al_syn"), 9900
    if case in ("grid_pair", "grid_syn"):
        return ng.sparse_large(seed=97, n_e=1600, n_i=400), psst.MODE_GRID, int(case == "grid_syn"), 300
    return ng.independent(2000, seed=98, n_nets=2, rate_hz=200.0), psst.MODE_CTA, 0, 1990


def _run(spec, mode, gate_mode, step0, chunks, y0=None, graph=False, **kw):
    from paper_1906_03958_gb300 import psst
    with psst.Network(spec, init_state=y0, mode=mode, gate_mode=gate_mode, rec_stride=3, rec_capacity=200,
                      **kw) as net:
        net.set_graph_mode(graph)
        net.set_step(step0)
        for c in chunks:
            net.integrate(c)
        net.status()
        return net.get_state_numpy(), net.read_record()


CASES = ["al_pair", "al_syn", "grid_pair", "grid_syn", "indep"]


@pytest.mark.parametrize("case", CASES)
def test_classic_and_one_stage_tableaus_are_rk4_and_euler_bitwise(case):
    from paper_1906_03958_gb300 import psst
    spec, mode, gm, step0 = _case(case)
    for tab, method in ((RK4, psst.METHOD_RK4), (EULER, psst.METHOD_EULER)):
        a = _run(spec, mode, gm, step0, [57, 64], method=method)
        b = _run(spec, mode, gm, step0, [57, 64], tableau=tab)
        np.testing.assert_array_equal(a[0], b[0])
        np.testing.assert_array_equal(a[1], b[1])


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("tab", [MIDPOINT, HEUN3, RALSTON2], ids=["midpoint", "heun3", "ralston2"])
def test_tableau_single_step_error(case, tab):
    from paper_1906_03958_gb300 import psst
    spec, mode, gm, step0 = _case(case)
    N, S = spec.n_neurons, spec.n_synapses
    y32 = oracle.integrate(spec, oracle.rest_state(spec), 40, step0=step0, tableau=tab)[0].astype(np.float32)
    y64, _ = oracle.integrate(spec, y32.astype(np.float64), 1, step0=step0 + 40, tableau=tab)
    with psst.Network(spec, init_state=y32, mode=mode, gate_mode=gm, tableau=tab) as net:
        net.set_step(step0 + 40)
        net.integrate(1)
        net.status()
        got = net.get_state_numpy()
    assert step_error(got, y64, N, S) <= STEP_TOL


@pytest.mark.parametrize("gate_mode", [0, 1])
def test_tableau_cta_equals_grid_chunked_and_graph_bitwise(gate_mode):
    # three stages per step: the stage parity runs on across steps, and odd
    # step counts leave the grid's final gate maps in table 1 (the same work
    # items in both modes, so that the synaptic sums group alike)
    from paper_1906_03958_gb300 import psst
    spec = ng.antennal_lobe(seed=99)
    y0 = oracle.rest_state(spec).astype(np.float32)
    out = [_run(spec, m, gate_mode, 9900, ch, y0=y0, graph=g, tableau=HEUN3, item_chunks=2)
           for m, ch, g in ((psst.MODE_CTA, [301], False), (psst.MODE_GRID, [301], False),
                            (psst.MODE_GRID, [100, 101, 100], False), (psst.MODE_CTA, [100, 100, 101], False),
                            (psst.MODE_CTA, [43] * 7, True))]
    for y, rec in out[1:]:
        np.testing.assert_array_equal(y, out[0][0])
        np.testing.assert_array_equal(rec, out[0][1])
    assert np.ptp(out[0][0][:spec.n_neurons]) > 10.0


@pytest.mark.parametrize("tab,sets", [(HEUN3, 1), (MIDPOINT, 3)], ids=["heun3", "midpoint-batch"])
def test_tableau_adjoint_matches_oracle(tab, sets):
    import torch
    from paper_1906_03958_gb300 import psst
    _, spec = ng.differentiated(n_sets=sets, seed=100 + sets, n_pn=12, n_ln=4)
    spec.pulse_on[:] = 5
    spec.pulse_off[:] = 10_000
    rng = np.random.default_rng(sets)
    nsteps, stride = 600, 6
    g = rng.standard_normal((nsteps // stride, spec.n_neurons))
    gy64, gw64, gp64 = oracle.adjoint(spec, oracle.rest_state(spec), nsteps, g, stride, ckpt=64, tableau=tab)
    with psst.Network(spec, rec_stride=stride, rec_capacity=nsteps // stride + 1, tableau=tab) as net:
        res = [net.adjoint(nsteps, torch.from_numpy(g.astype(np.float32)).cuda(), ck) for ck in (64, 7)]
        net.status()
    gw, gp, gy = (x.cpu().numpy() for x in res[0])
    for b in range(spec.n_nets):
        s0, s1 = spec.row_ptr[spec.net_neuron_off[b]], spec.row_ptr[spec.net_neuron_off[b + 1]]
        assert grad_error(gw[s0:s1], gw64[s0:s1]) <= GRAD_TOL
        assert grad_error(gp[2 * b:2 * b + 2], gp64[2 * b:2 * b + 2]) <= GRAD_TOL
    assert grad_error(gy.ravel(), gy64[:4 * spec.n_neurons]) <= GRAD_TOL
    for x, y in zip(res[1], res[0]):
        assert grad_error(x.cpu().numpy(), y.cpu().numpy()) <= 1e-5
