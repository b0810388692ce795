"""Networks without synapses (independent HH neurons, the paper's Fig. 2b
systems): integrated one thread per neuron with no barriers, against the
oracle and, bitwise, against the coupled kernels on the same neurons."""
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


def test_independent_single_step_error_with_noise_and_pulse():
    spec = ng.independent(3000, seed=71, n_nets=3, rate_hz=200.0)
    N, S = spec.n_neurons, spec.n_synapses
    y32 = oracle.integrate(spec, oracle.rest_state(spec), 40, step0=1990)[0].astype(np.float32)
    y64, _ = oracle.integrate(spec, y32.astype(np.float64), 1, step0=2030)
    with _net(spec, init_state=y32) as net:
        info = net.info()
        assert info["n_independent_nets"] == 3 and info["n_launch_classes"] == 0
        net.set_step(2030)
        net.integrate(1)
        net.status()
        assert net.info()["kernel_launches"] == 1
        got = net.get_state_numpy()
    assert step_error(got, y64, N, S) <= STEP_TOL


def test_independent_equals_coupled_kernel_bitwise():
    # the same neurons, once without synapses and once with one synapse of
    # weight 0 each (coupled kernel, zero synaptic current): same neuron
    # state and record, bit for bit
    base = ng.independent(600, seed=72, n_nets=2, rate_hz=100.0)
    N = base.n_neurons
    half = N // 2
    post = np.arange(N)
    pre_local = np.where(post < half, (post + 1) % half, (post - half + 1) % (N - half))
    coupled = ng.NetworkSpec(
        net_neuron_off=base.net_neuron_off, neuron_type=base.neuron_type, neuron_params=base.neuron_params,
        row_ptr=np.arange(N + 1, dtype=np.int64), pre=pre_local.astype(np.int32),
        weight=np.zeros(N, np.float32), syn_type=np.zeros(N, np.int32), syn_params=base.syn_params,
        i_const=base.i_const, pulse_amp=base.pulse_amp, pulse_on=base.pulse_on, pulse_off=base.pulse_off,
        noise_seed=base.noise_seed, noise_thresh=base.noise_thresh, noise_amp=base.noise_amp, dt=base.dt,
        name="independent+zero-weight synapses")
    out = []
    for spec in (base, coupled):
        with _net(spec, rec_stride=7, rec_capacity=200) as net:
            assert net.info()["n_independent_nets"] == (2 if spec is base else 0)
            net.set_step(1500)
            net.integrate(700)
            net.status()
            out.append((net.get_state_numpy()[:4 * N], net.read_record()))
    np.testing.assert_array_equal(out[0][0], out[1][0])
    np.testing.assert_array_equal(out[0][1], out[1][1])
    assert np.ptp(out[0][0][:N]) > 10.0  # some neurons spike


def test_mixed_batch_equals_alone_and_graph_replay():
    # independent networks beside coupled ones (own stream), chunked and
    # replayed through a CUDA graph: each network as when integrated alone
    mixed = ng.concat_specs([ng.independent(500, seed=73, n_nets=2), ng.plain20(seed=74),
                             ng.independent(300, seed=75)])
    with _net(mixed, rec_stride=10, rec_capacity=100) as net:
        assert net.info()["n_independent_nets"] == 3
        net.set_graph_mode(True)
        for _ in range(4):
            net.integrate(150)
        net.status()
        y = net.get_state_numpy()
        rec = net.read_record()
    N = mixed.n_neurons
    for b in range(mixed.n_nets):
        alone = mixed.subset([b])
        n0, n1 = int(mixed.net_neuron_off[b]), int(mixed.net_neuron_off[b + 1])
        with _net(alone, rec_stride=10, rec_capacity=100) as one:
            one.integrate(600)
            one.status()
            ya = one.get_state_numpy()
            ra = one.read_record()
        na = alone.n_neurons
        for x in range(4):
            np.testing.assert_array_equal(y[x * N + n0:x * N + n1], ya[x * na:(x + 1) * na])
        np.testing.assert_array_equal(rec[:, n0:n1], ra)
