"""Parity of the CUDA path (through the C interface) with the FP64 oracle.

Bars (floating point):
  * one RK4 step from an identical FP32 state: relative error <= 1e-5 with
    floors of 1 mV for V and 1e-3 for gates (tests.helpers.step_error);
  * spike times within 0.05 ms over 100 ms on a non-chaotic network;
  * bitwise identity between GPU runs that must agree exactly (chunked vs
    whole, batched vs alone, record ring vs state).
Integer decisions (noise events) must match exactly.
"""
import numpy as np
import pytest

import oracle
from paper_1906_03958_gb300 import netgen as ng
from tests.helpers import step_error

pytestmark = pytest.mark.gpu

STEP_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    from paper_1906_03958_gb300 import psst
    assert torch.cuda.is_available()
    psst.load()


def _net(spec, **kw):
    from paper_1906_03958_gb300 import psst
    return psst.Network(spec, **kw)


def _gpu_one_step(spec, y32, step, **kw):
    with _net(spec, init_state=y32, **kw) as net:
        net.set_step(step)
        net.integrate(1)
        net.status()
        return net.get_state_numpy()


def _states_along_oracle(spec, steps, step0=0):
    """FP32 states visited by the oracle at the given step indices."""
    y = oracle.rest_state(spec)
    net = oracle.OracleNet(spec)
    out, k = [], step0
    for s in steps:
        y, _ = oracle.integrate(net, y, s - k, step0=k)
        k = s
        out.append((s, y.astype(np.float32)))
    return out


@pytest.mark.parametrize("name,spec_fn,steps", [
    ("plain20", lambda: ng.plain20(), [0, 150, 420, 1000]),
    ("antennal_lobe", lambda: ng.antennal_lobe(), [9995, 10005, 10130]),
])
def test_single_step_error(name, spec_fn, steps):
    spec = spec_fn()
    N, S = spec.n_neurons, spec.n_synapses
    onet = oracle.OracleNet(spec)
    worst = 0.0
    for step, y32 in _states_along_oracle(spec, steps, step0=steps[0]):
        y64, _ = oracle.integrate(onet, y32.astype(np.float64), 1, step0=step)
        got = _gpu_one_step(spec, y32, step)
        worst = max(worst, step_error(got, y64, N, S))
    assert worst <= STEP_TOL, worst


def test_single_step_error_random_states():
    # random (non-physiological) states exercise every branch of the rates,
    # including the removable singularities at -40 and -55 mV
    spec = ng.antennal_lobe(seed=7)
    N, S = spec.n_neurons, spec.n_synapses
    rng = np.random.default_rng(0)
    y = np.zeros(4 * N + 2 * S, np.float32)
    y[:N] = rng.uniform(-90, 50, N)
    y[:8] = [-40.0, -55.0, -40.0004, -54.9996, -39.5, -55.5, 49.0, -89.0]
    y[N:4 * N] = rng.uniform(0, 1, 3 * N)
    y[4 * N:] = rng.uniform(0, 1, 2 * S)
    y[4 * N + S:] *= 5.0  # GABA_B s ranges over ~0..5
    y64, _ = oracle.integrate(spec, y.astype(np.float64), 1, step0=12345)
    got = _gpu_one_step(spec, y, 12345)
    assert step_error(got, y64, N, S) <= STEP_TOL


def test_spike_times_non_chaotic():
    # plain 20-neuron network with weights x0.1 (1-7 spikes per neuron):
    # spike times within 0.05 ms of the FP64 oracle over 100 ms
    spec = ng.plain20(weight_scale=0.1)
    y0 = oracle.rest_state(spec)
    _, rec64 = oracle.integrate(spec, y0, 10000, rec_stride=1)
    with _net(spec, init_state=y0.astype(np.float32), rec_stride=1, rec_capacity=10000) as net:
        net.integrate(10000)
        net.status()
        rec32 = net.read_record()
    assert rec32.shape == rec64.shape
    t64 = oracle.spike_times(rec64, 0.01)
    t32 = oracle.spike_times(rec32, 0.01)
    n_spikes = 0
    for a, b in zip(t64, t32):
        assert len(a) == len(b)
        if len(a):
            assert np.max(np.abs(a - b)) < 0.05
        n_spikes += len(a)
    assert n_spikes >= 20


def test_chunked_equals_whole_bitwise():
    spec = ng.antennal_lobe()
    y0 = oracle.rest_state(spec).astype(np.float32)
    with _net(spec, init_state=y0, rec_stride=7, rec_capacity=200) as a, \
            _net(spec, init_state=y0, rec_stride=7, rec_capacity=200) as b:
        a.set_step(9900), b.set_step(9900)
        a.integrate(1000)
        for n in (1, 299, 77, 623):
            b.integrate(n)
        a.status(), b.status()
        np.testing.assert_array_equal(a.get_state_numpy(), b.get_state_numpy())
        np.testing.assert_array_equal(a.read_record(), b.read_record())


def test_set_state_restarts_the_compensated_sums():
    # The step sums carry each state variable's rounding remainder across
    # steps and calls; get_state returns the FP32 values and set_state starts
    # the remainders at zero, so a handle continuing from a copied state
    # agrees with the uninterrupted run far below the single-step bar, and two
    # handles given the same state continue bit for bit
    spec = ng.antennal_lobe()
    N, S = spec.n_neurons, spec.n_synapses
    y0 = oracle.rest_state(spec).astype(np.float32)
    with _net(spec, init_state=y0) as a:
        a.set_step(9900)
        a.integrate(700)
        y = a.get_state_numpy()
        with _net(spec, init_state=y) as b:
            b.set_step(10600)
            a.integrate(300)
            b.integrate(300)
            a.status(), b.status()
            assert step_error(b.get_state_numpy(), a.get_state_numpy(), N, S) <= 1e-5
            yb = b.get_state().clone()
            a.set_state(yb)
            b.set_state(yb)
            a.integrate(200)
            b.integrate(200)
            a.status(), b.status()
            np.testing.assert_array_equal(a.get_state_numpy(), b.get_state_numpy())


def test_batched_equals_alone_bitwise():
    specs = [ng.antennal_lobe(seed=21, n_pn=30, n_ln=10), ng.antennal_lobe(seed=22),
             ng.antennal_lobe(seed=23, n_pn=12, n_ln=4, p=0.3)]
    both = ng.concat_specs(specs)
    y0s = [oracle.rest_state(s).astype(np.float32) for s in specs]
    # batch state: V, m, h, n blocks and r, s blocks concatenated per network
    Ns = [s.n_neurons for s in specs]
    Ss = [s.n_synapses for s in specs]
    parts = []
    for blk in range(4):
        parts += [y[blk * n:(blk + 1) * n] for y, n in zip(y0s, Ns)]
    for blk in range(2):
        parts += [y[4 * n + blk * s:4 * n + (blk + 1) * s] for y, n, s in zip(y0s, Ns, Ss)]
    yb = np.concatenate(parts)
    kw = dict(block_threads=256, item_chunks=3)
    with _net(both, init_state=yb, **kw) as nb:
        nb.integrate(500)
        nb.status()
        got = nb.get_state_numpy()
    off_n, off_s = 0, 0
    Nt, St = sum(Ns), sum(Ss)
    for s, y0, n, sy in zip(specs, y0s, Ns, Ss):
        with _net(s, init_state=y0, **kw) as na:
            na.integrate(500)
            na.status()
            alone = na.get_state_numpy()
        for blk in range(4):
            np.testing.assert_array_equal(got[blk * Nt + off_n:blk * Nt + off_n + n], alone[blk * n:(blk + 1) * n])
        for blk in range(2):
            np.testing.assert_array_equal(got[4 * Nt + blk * St + off_s:4 * Nt + blk * St + off_s + sy],
                                          alone[4 * n + blk * sy:4 * n + (blk + 1) * sy])
        off_n += n
        off_s += sy


def test_ragged_batch_single_step():
    # several CTAs' worth of networks of uneven size, incl. a ragged tail of
    # tiny ones, and networks too large for one SM (cluster of CTAs)
    small = ng.batched(n_nets=40, base_seed=900, n_min=2, n_max=120)
    big = ng.batched(n_nets=3, base_seed=950, n_min=290, n_max=300)
    spec = ng.concat_specs([small, big])
    N, S = spec.n_neurons, spec.n_synapses
    onet = oracle.OracleNet(spec)
    for step, y32 in _states_along_oracle(spec, [0, 300]):
        y64, _ = oracle.integrate(onet, y32.astype(np.float64), 1, step0=step)
        with _net(spec, init_state=y32, block_threads=256) as net:
            info = net.info()
            net.set_step(step)
            net.integrate(1)
            net.status()
            got = net.get_state_numpy()
        assert info["n_cluster_nets"] >= 1 and info["n_single_cta_nets"] >= 40
        assert step_error(got, y64, N, S) <= STEP_TOL


@pytest.mark.parametrize("block,G", [(32, 1), (128, 4), (1024, 16), (64, 64), (256, 7)])
def test_launch_shapes(block, G):
    spec = ng.antennal_lobe(seed=5)
    N, S = spec.n_neurons, spec.n_synapses
    (step, y32), = _states_along_oracle(spec, [10050], step0=9990)
    y64, _ = oracle.integrate(spec, y32.astype(np.float64), 1, step0=step)
    got = _gpu_one_step(spec, y32, step, block_threads=block, item_chunks=G)
    assert step_error(got, y64, N, S) <= STEP_TOL


def test_multi_step_short_horizon():
    # 200 steps through a spike volley: trajectory stays close to the oracle
    spec = ng.plain20()
    y0 = oracle.rest_state(spec)
    _, rec64 = oracle.integrate(spec, y0, 200, rec_stride=1)
    with _net(spec, init_state=y0.astype(np.float32), rec_stride=1, rec_capacity=200) as net:
        net.integrate(200)
        net.status()
        rec32 = net.read_record()
    assert np.max(np.abs(rec32 - rec64)) < 1e-2


def test_noise_events_bit_exact():
    # passive neurons: each noise event adds exactly amp*dt/C, so any
    # mismatched event decision shows up as a jump of 2e-2 mV
    passive = dict(ng.HH, gNa=0.0, gK=0.0, gL=0.0, gKL=0.0)
    thresh = int(0.05 * (1 << 24))
    n = 300
    spec = ng.single_network(np.zeros(n), np.zeros(n), [], [], [], [], ng.neuron_table(passive),
                             ng.synapse_table(ng.ACH), noise_seed=0xDEADBEEF12345, noise_thresh=thresh,
                             noise_amp=2.0)
    y0 = oracle.rest_state(spec)
    y64, _ = oracle.integrate(spec, y0, 400, step0=(1 << 32) - 200)
    with _net(spec, init_state=y0.astype(np.float32)) as net:
        net.set_step((1 << 32) - 200)
        net.integrate(400)
        net.status()
        got = net.get_state_numpy()
    assert np.max(np.abs(got[:n] - y64[:n])) < 2e-3
    assert np.ptp(y64[:n]) > 0.1  # events happened


def test_pulse_edges_and_record_ring():
    passive = dict(ng.HH, gNa=0.0, gK=0.0, gL=0.0, gKL=0.0)
    spec = ng.single_network([0, 0], [0.5, 0.0], [], [], [], [], ng.neuron_table(passive),
                             ng.synapse_table(ng.ACH), pulse_amp=[3.0, -1.0], pulse_on=7, pulse_off=19)
    y0 = oracle.rest_state(spec)
    _, rec64 = oracle.integrate(spec, y0, 40, rec_stride=3)
    with _net(spec, init_state=y0.astype(np.float32), rec_stride=3, rec_capacity=5) as net:
        net.integrate(17)
        net.integrate(23)
        net.status()
        rec32 = net.read_record()
        assert net.info()["rec_frames"] == 13
    assert rec32.shape == (5, 2)
    np.testing.assert_allclose(rec32, rec64[-5:], rtol=0, atol=2e-4)


def test_state_roundtrip_and_zero_steps():
    import torch
    spec = ng.plain20()
    with _net(spec) as net:
        y = net.get_state()  # rest state built by the library
        y64 = oracle.rest_state(spec)
        np.testing.assert_allclose(y.cpu().numpy(), y64, rtol=1e-6, atol=1e-7)
        net.integrate(0)
        np.testing.assert_array_equal(net.get_state().cpu().numpy(), y.cpu().numpy())
        z = torch.linspace(0, 1, net.dim, device="cuda")
        net.set_state(z)
        np.testing.assert_array_equal(net.get_state().cpu().numpy(), z.cpu().numpy())


def test_edge_networks_single_neuron_and_no_synapses():
    # a lone neuron, a network without synapses and a 2-neuron network in one batch
    lone = ng.single_network([0], [10.0], [], [], [], [], ng.neuron_table(ng.HH), ng.synapse_table(ng.ACH))
    nosyn = ng.single_network([0] * 5, np.linspace(0, 12, 5), [], [], [], [], ng.neuron_table(ng.HH),
                              ng.synapse_table(ng.ACH))
    pair = ng.single_network([0, 0], [10.0, 0.0], [1], [0], [0.5], [0], ng.neuron_table(ng.HH),
                             ng.synapse_table(ng.ACH))
    spec = ng.concat_specs([lone, nosyn, pair])
    N, S = spec.n_neurons, spec.n_synapses
    y0 = oracle.rest_state(spec)
    y64, rec64 = oracle.integrate(spec, y0, 3000, rec_stride=10)
    with _net(spec, init_state=y0.astype(np.float32), rec_stride=10, rec_capacity=300) as net:
        net.integrate(3000)
        net.status()
        rec32 = net.read_record()
    t64 = oracle.spike_times(rec64, 0.1)
    t32 = oracle.spike_times(rec32, 0.1)
    for a, b in zip(t64, t32):
        assert len(a) == len(b)
        if len(a):
            assert np.max(np.abs(a - b)) < 0.05


def test_nonfinite_state_is_reported():
    from paper_1906_03958_gb300 import psst
    spec = ng.plain20()
    with _net(spec) as net:
        y = net.get_state_numpy()
        y[3] = np.nan
        net.set_state(y)
        net.integrate(5)
        with pytest.raises(psst.PsstError) as ei:
            net.status()
        assert ei.value.code == -4
        net.status()  # cleared after being read


def test_psst_sync_reports_device_errors_from_integrate(monkeypatch):
    # PSST_SYNC: psst_integrate waits and returns the device error itself
    from paper_1906_03958_gb300 import psst
    spec = ng.plain20()
    with _net(spec) as net:
        y = net.get_state_numpy()
        y[3] = np.nan
        net.set_state(y)
        monkeypatch.setenv("PSST_SYNC", "1")
        with pytest.raises(psst.PsstError) as ei:
            net.integrate(5)
        assert ei.value.code == -4
        net.set_state(np.nan_to_num(y, nan=-65.0))
        net.integrate(5)  # no error: returns 0 after synchronising
        monkeypatch.setenv("PSST_SYNC", "0")
        net.integrate(5)
        net.status()


def test_graph_replay_bitwise_equal_to_direct_launches():
    spec = ng.concat_specs([ng.antennal_lobe(seed=51), ng.antennal_lobe(seed=52, n_pn=30, n_ln=10)])
    y0 = oracle.rest_state(spec).astype(np.float32)
    with _net(spec, init_state=y0, rec_stride=10, rec_capacity=100) as a, \
            _net(spec, init_state=y0, rec_stride=10, rec_capacity=100) as b:
        a.set_step(9950), b.set_step(9950)
        b.set_graph_mode(True)
        a.integrate(300)
        for _ in range(3):
            b.integrate(100)  # captured once, replayed twice with new step indices
        a.status(), b.status()
        np.testing.assert_array_equal(a.get_state_numpy(), b.get_state_numpy())
        np.testing.assert_array_equal(a.read_record(), b.read_record())


@pytest.mark.parametrize("item_chunks", [2, 0])
def test_autotune_keeps_results_bitwise(item_chunks):
    # 24 networks need few SMs, so the tuner also tries larger clusters
    spec = ng.batched(n_nets=24, base_seed=700, n_min=20, n_max=300)
    y0 = oracle.rest_state(spec).astype(np.float32)
    with _net(spec, init_state=y0, item_chunks=item_chunks) as a, \
            _net(spec, init_state=y0, item_chunks=item_chunks) as b:
        b.autotune(50)
        np.testing.assert_array_equal(b.get_state_numpy(), y0)  # state restored
        a.integrate(200)
        b.integrate(200)
        a.status(), b.status()
        np.testing.assert_array_equal(a.get_state_numpy(), b.get_state_numpy())


@pytest.mark.parametrize("gate_mode", [0, 1])
def test_forced_cluster_sizes_agree_bitwise(gate_mode):
    # the antennal lobe and a small batch on clusters of at least 1, 2 and 4
    # CTAs, and as the tuner chooses: the same results bit for bit
    spec = ng.concat_specs([ng.antennal_lobe(seed=91), ng.antennal_lobe(seed=92, n_pn=45, n_ln=15)])
    y0 = oracle.rest_state(spec).astype(np.float32)
    out = []
    for mc, tune in ((1, False), (2, False), (4, False), (0, True)):
        with _net(spec, init_state=y0, rec_stride=10, rec_capacity=50, min_cluster=mc, gate_mode=gate_mode) as net:
            if tune:
                net.autotune(100)
            info = net.info()
            if mc > 1:
                assert info["n_cluster_nets"] == 2 and info["n_single_cta_nets"] == 0
            net.set_step(9800)
            net.integrate(400)
            net.status()
            out.append((net.get_state_numpy(), net.read_record()))
    for y, rec in out[1:]:
        np.testing.assert_array_equal(y, out[0][0])
        np.testing.assert_array_equal(rec, out[0][1])


def test_pair_gates_agree_with_per_synapse_gates():
    # one gate per (presynaptic neuron, type) pair and one per synapse reach
    # the same RK4 map; only the summation grouping of the synaptic current
    # differs (typed items), so both meet the single-step bound against the
    # oracle and stay together over a short horizon
    from paper_1906_03958_gb300 import psst
    specs = [ng.antennal_lobe(seed=61), ng.antennal_lobe(seed=62, n_pn=40, n_ln=20)]
    spec = ng.concat_specs(specs)
    N, S = spec.n_neurons, spec.n_synapses
    y32 = oracle.integrate(spec, oracle.rest_state(spec), 40, step0=9900)[0].astype(np.float32)
    y64, _ = oracle.integrate(spec, y32.astype(np.float64), 1, step0=9940)
    traj = []
    for gm in (0, 1):
        with _net(spec, init_state=y32, gate_mode=gm, rec_stride=20, rec_capacity=100) as net:
            assert net.info()["n_pair_gate_nets"] == (2 if gm == 0 else 0)
            net.set_step(9940)
            net.integrate(1)
            net.status()
            assert step_error(net.get_state_numpy(), y64, N, S) <= STEP_TOL
            net.integrate(299)
            net.status()
            traj.append(net.read_record())
    np.testing.assert_allclose(traj[0], traj[1], rtol=0, atol=1e-3)


def test_set_state_switches_gate_layout():
    # a state whose pair gates differ must leave the per-pair layout; results
    # then equal a network that always runs per synapse
    spec = ng.antennal_lobe(seed=63)
    N = spec.n_neurons
    y = oracle.rest_state(spec).astype(np.float32)
    y[4 * N:4 * N + spec.n_synapses] = np.random.default_rng(0).uniform(0, 1, spec.n_synapses)
    with _net(spec) as a, _net(spec, gate_mode=1) as b:
        a.integrate(10)          # per-pair layout from rest
        a.set_state(y)
        b.set_state(y)
        a.set_step(0), b.set_step(0)
        a.integrate(200)
        b.integrate(200)
        a.status(), b.status()
        np.testing.assert_array_equal(a.get_state_numpy(), b.get_state_numpy())


def test_torch_allocator_serves_the_handle():
    # device memory from PyTorch's caching allocator through psst_allocator:
    # same results, memory visible to torch while the handle lives
    import torch
    spec = ng.concat_specs([ng.antennal_lobe(seed=95), ng.antennal_lobe(seed=96, n_pn=30, n_ln=10)])
    y0 = oracle.rest_state(spec).astype(np.float32)
    before = torch.cuda.memory_allocated()
    with _net(spec, init_state=y0, rec_stride=10, rec_capacity=50, allocator="torch") as a:
        assert a._allocator.blocks and torch.cuda.memory_allocated() > before
        a.set_step(9900)
        a.integrate(300)
        a.status()
        got = a.get_state_numpy(), a.read_record()
        alloc = a._allocator
    assert not alloc.blocks  # every block handed back at destroy
    with _net(spec, init_state=y0, rec_stride=10, rec_capacity=50) as b:
        b.set_step(9900)
        b.integrate(300)
        b.status()
        np.testing.assert_array_equal(got[0], b.get_state_numpy())
        np.testing.assert_array_equal(got[1], b.read_record())
