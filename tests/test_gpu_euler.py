"""Forward Euler (the paper's first-order method, Eq. euler) on the GPU against
the oracle's Euler step, in every execution path, and its bitwise
consistency between paths and launch forms."""
import numpy as np
import pytest

import oracle
from paper_1906_03958_gb300 import netgen as ng
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


def test_adjoint_requires_rk4():
    import torch
    from paper_1906_03958_gb300 import psst
    spec = ng.antennal_lobe(seed=86, n_pn=12, n_ln=4)
    with _net(spec, rec_stride=1, rec_capacity=10) as net:
        net.integrate(10)
        with pytest.raises(psst.PsstError) as ei:
            net.adjoint(10, torch.zeros((10, spec.n_neurons), device="cuda"), 5)
        assert ei.value.code == -7
