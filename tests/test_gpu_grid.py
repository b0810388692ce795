"""Grid-wide mode (one large sparse network over all SMs) against the oracle,
against the CTA mode, and its bounded device-wide barrier."""
import numpy as np
import pytest

import oracle
from paper_1906_03958_gb300 import netgen as ng
from tests.helpers import step_error

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-5


def _net(spec, **kw):
    from paper_1906_03958_gb300 import psst
    return psst.Network(spec, **kw)


def _mid_sparse(seed=31, noise=True):
    return ng.sparse_large(seed=seed, n_e=1600, n_i=400, p=0.02,
                           rate_hz=20.0 if noise else 0.0)


def _oracle_state(spec, nsteps, step0=0):
    y, _ = oracle.integrate(spec, oracle.rest_state(spec), nsteps, step0=step0)
    return y.astype(np.float32)


def test_grid_single_step_error():
    from paper_1906_03958_gb300 import psst
    spec = _mid_sparse()
    N, S = spec.n_neurons, spec.n_synapses
    for step0, n in ((0, 0), (0, 60)):
        y32 = _oracle_state(spec, n, step0)
        y64, _ = oracle.integrate(spec, y32.astype(np.float64), 1, step0=step0 + n)
        with _net(spec, init_state=y32, mode=psst.MODE_GRID) as net:
            info = net.info()
            net.set_step(step0 + n)
            net.integrate(1)
            net.status()
            got = net.get_state_numpy()
        assert info["mode"] == psst.MODE_GRID and info["grid_ctas"] > 100
        assert step_error(got, y64, N, S) <= STEP_TOL


@pytest.mark.parametrize("gate_mode", [0, 1])
def test_grid_equals_cta_mode_bitwise(gate_mode):
    # dense-in-one-CTA and spread-over-the-GPU evaluate the same per-row sums
    # in the same order, so the two representations agree exactly (both gate
    # layouts, with second-order GABA_B gates)
    from paper_1906_03958_gb300 import psst
    spec = ng.antennal_lobe(seed=41)
    y0 = oracle.rest_state(spec).astype(np.float32)
    out = []
    for mode in (psst.MODE_CTA, psst.MODE_GRID):
        with _net(spec, init_state=y0, mode=mode, block_threads=256, item_chunks=2,
                  rec_stride=5, rec_capacity=100, gate_mode=gate_mode) as net:
            net.set_step(9950)
            net.integrate(300)
            net.status()
            out.append((net.get_state_numpy(), net.read_record()))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])


def test_grid_chunked_equals_whole_bitwise():
    from paper_1906_03958_gb300 import psst
    spec = _mid_sparse(seed=32)
    y0 = oracle.rest_state(spec).astype(np.float32)
    with _net(spec, init_state=y0, mode=psst.MODE_GRID) as a, _net(spec, init_state=y0, mode=psst.MODE_GRID) as b:
        a.integrate(200)
        b.integrate(13)
        b.integrate(187)
        a.status(), b.status()
        np.testing.assert_array_equal(a.get_state_numpy(), b.get_state_numpy())


def test_grid_trajectory_with_noise_short_horizon():
    from paper_1906_03958_gb300 import psst
    spec = _mid_sparse(seed=33)
    y0 = oracle.rest_state(spec)
    _, rec64 = oracle.integrate(spec, y0, 100, rec_stride=10)
    with _net(spec, init_state=y0.astype(np.float32), mode=psst.MODE_GRID, rec_stride=10, rec_capacity=10) as net:
        net.integrate(100)
        net.status()
        rec32 = net.read_record()
    assert np.max(np.abs(rec32 - rec64)) < 1e-2


def test_sparse_large_full_size_single_step():
    # the full 10,000-neuron / ~2M-synapse network with shot noise
    from paper_1906_03958_gb300 import psst
    spec = ng.sparse_large()
    N, S = spec.n_neurons, spec.n_synapses
    y32 = oracle.rest_state(spec).astype(np.float32)
    y64, _ = oracle.integrate(spec, y32.astype(np.float64), 1, step0=777)
    with _net(spec, init_state=y32) as net:
        assert net.info()["mode"] == psst.MODE_GRID
        assert net.info()["n_pair_gate_nets"] == 1  # the compact gate table fits next to the items
        net.set_step(777)
        net.integrate(1)
        net.status()
        got = net.get_state_numpy()
    assert step_error(got, y64, N, S) <= STEP_TOL


def test_barrier_timeout_is_reported_and_recoverable():
    # a zero time limit makes every barrier wait give up at once: the kernel
    # records TIMEOUT and returns; the context stays usable afterwards
    from paper_1906_03958_gb300 import psst
    spec = _mid_sparse(seed=34, noise=False)
    y0 = oracle.rest_state(spec).astype(np.float32)
    with _net(spec, init_state=y0, mode=psst.MODE_GRID) as net:
        net.set_barrier_timeout(0)
        net.integrate(50)
        with pytest.raises(psst.PsstError) as ei:
            net.status()
        assert ei.value.code == -5
        net.set_barrier_timeout(2_000_000_000)
        net.set_state(y0)
        net.set_step(0)
        net.integrate(20)
        net.status()
        got = net.get_state_numpy()
    with _net(spec, init_state=y0, mode=psst.MODE_GRID) as ref:
        ref.integrate(20)
        ref.status()
        np.testing.assert_array_equal(got, ref.get_state_numpy())


def test_grid_pair_gates_agree_with_per_synapse_gates():
    # the compact per-pair gate table and one gate per synapse: both meet the
    # single-step bound against the oracle (with noise) and stay together
    # over a short horizon
    from paper_1906_03958_gb300 import psst
    spec = _mid_sparse(seed=35)
    N, S = spec.n_neurons, spec.n_synapses
    y32 = _oracle_state(spec, 30, 4300)
    y64, _ = oracle.integrate(spec, y32.astype(np.float64), 1, step0=4330)
    traj = []
    for gm in (0, 1):
        with _net(spec, init_state=y32, mode=psst.MODE_GRID, gate_mode=gm, rec_stride=7, rec_capacity=100) as net:
            assert net.info()["n_pair_gate_nets"] == (1 if gm == 0 else 0)
            net.set_step(4330)
            net.integrate(1)
            net.status()
            assert step_error(net.get_state_numpy(), y64, N, S) <= STEP_TOL
            net.integrate(299)
            net.status()
            traj.append(net.read_record())
    np.testing.assert_allclose(traj[0], traj[1], rtol=0, atol=1e-3)


def test_grid_set_state_switches_gate_layout():
    # unequal gates within a pair force one gate per synapse; a state with
    # equal pair gates brings the per-pair table back
    from paper_1906_03958_gb300 import psst
    spec = _mid_sparse(seed=36, noise=False)
    N, S = spec.n_neurons, spec.n_synapses
    rest = oracle.rest_state(spec).astype(np.float32)
    y = rest.copy()
    y[4 * N:4 * N + S] = np.random.default_rng(1).uniform(0, 1, S)
    with _net(spec, mode=psst.MODE_GRID) as a, _net(spec, mode=psst.MODE_GRID, gate_mode=1) as b:
        assert a.info()["n_pair_gate_nets"] == 1
        a.integrate(10)
        a.set_state(y)
        b.set_state(y)
        assert a.info()["n_pair_gate_nets"] == 0
        a.set_step(0), b.set_step(0)
        a.integrate(150)
        b.integrate(150)
        a.status(), b.status()
        np.testing.assert_array_equal(a.get_state_numpy(), b.get_state_numpy())
        a.set_state(rest)
        assert a.info()["n_pair_gate_nets"] == 1
