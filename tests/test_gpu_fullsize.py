"""Parity at the benchmarked sizes.

* The differentiated workload at full size: one parameter set of the
  120-neuron antennal-lobe network (dense 120 x 120 weights plus the GABA_B
  block), 20,000 RK4 steps, checkpoints every 1,000 steps recorded by the
  forward (the benchmark's path) and the adjoint's own checkpointing: FP32
  gradients of the mean-square PN trace loss (targets at the hidden
  parameters) against the FP64 oracle's adjoint (every weight, every table
  entry, the initial-state adjoint) and against FP64 central differences on
  10 coordinates.  Expected values: tests/golden/adjoint_al120_20k.npz,
  written by tests/golden/make_adjoint_al120.py from the oracle alone.
* The 4,096-network batch exactly as the benchmark runs it (autotuned size
  classes and gate-table copies, CUDA-graph replay, V recorded every 10
  steps): one step from a seeded physiological state against the oracle's
  step, element by element.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1906_03958_gb300 import netgen as ng
from tests.golden import make_adjoint_al120 as gold
from tests.helpers import fd_reference, grad_error, step_error

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3
HERE = os.path.dirname(os.path.abspath(__file__))


def _check_against_golden(gw, gp, gy, G):
    assert grad_error(gw, G["gw"]) <= GRAD_TOL, grad_error(gw, G["gw"])
    assert grad_error(gp, G["gp"]) <= GRAD_TOL, grad_error(gp, G["gp"])
    if gy is not None:
        assert grad_error(gy.ravel(), G["gy0"]) <= GRAD_TOL, grad_error(gy.ravel(), G["gy0"])
    ref, err = fd_reference(G["fd"])
    ks, ps = list(G["fd_w_index"]), [tuple(p) for p in G["fd_p_index"]]
    got = [gw[k] for k in ks] + [gp[p] for p in ps]
    for c, (x, want, e) in enumerate(zip(got, ref, err)):
        assert abs(x - want) <= GRAD_TOL * abs(want) + e, (c, x, want, e)


@pytest.fixture(scope="module")
def golden():
    return np.load(os.path.join(HERE, "golden", "adjoint_al120_20k.npz"))


@pytest.fixture(scope="module")
def target():
    # the target traces at the hidden parameters, from the FP64 oracle (the
    # loss's data, not an expected value; about half a minute on one core)
    return gold.target_traces()


def test_differentiated_full_size_adjoint(golden, target):
    import torch
    from paper_1906_03958_gb300 import psst
    from paper_1906_03958_gb300.autograd import trace
    _, spec = gold.workload()
    T, K, npn = int(golden["nsteps"]), int(golden["ckpt"]), int(golden["n_pn"])
    N = spec.n_neurons
    vstar = torch.from_numpy(target.astype(np.float32)).cuda()
    # the benchmark's path: the forward records its checkpoints, the adjoint
    # uses them, with dL/dV from the GPU's own traces
    with psst.Network(spec, rec_stride=1, rec_capacity=T) as net:
        net.record_checkpoints(K, T)
        net.integrate(T)
        v = net.read_record(out=torch.empty((T, N), dtype=torch.float32, device="cuda"))
        dldv = torch.zeros_like(v)
        dldv[:, :npn] = 2.0 * (v[:, :npn] - vstar[:, :npn]) / (T * npn)
        rec = [x.cpu().numpy() for x in net.adjoint(T, dldv, 0)]
        net.status()
    loss32 = float(((v[:, :npn] - vstar[:, :npn]) ** 2).mean())
    assert abs(loss32 - float(golden["loss"])) <= 1e-4 * float(golden["loss"]), (loss32, float(golden["loss"]))
    _check_against_golden(rec[0], rec[1], rec[2], golden)
    # the torch.autograd path: mean-square loss, the adjoint's own checkpointing
    with psst.Network(spec, rec_stride=1, rec_capacity=T) as net:
        w = torch.from_numpy(spec.weight).cuda().requires_grad_(True)
        p = torch.from_numpy(spec.neuron_params).cuda().requires_grad_(True)
        v = trace(net, w, p, T, ckpt_every=K)
        loss = ((v[:, :npn] - vstar[:, :npn]) ** 2).mean()
        loss.backward()
    _check_against_golden(w.grad.cpu().numpy(), p.grad.cpu().numpy(), None, golden)


def _physiological_state(spec, seed):
    """A seeded state along the lines of a trajectory: V ~ U[-80, 40] mV
    (the spiking range), each gate m, h, n at its steady state (oracle) at a
    voltage within 10 mV of V, and synaptic gates r ~ U[0, 0.8],
    s ~ U[0, 0.5] drawn once per (presynaptic neuron, type) pair, so that
    every pair's gates are equal (the layout the benchmark runs)."""
    rng = np.random.default_rng(seed)
    N, S, nt = spec.n_neurons, spec.n_synapses, spec.syn_params.shape[0]
    y = np.empty(4 * N + 2 * S, np.float32)
    V = rng.uniform(-80.0, 40.0, N)
    y[:N] = V
    grid = np.arange(-95.0, 55.5, 0.5)
    table = np.array([oracle.steady_gates(u) for u in grid])  # [len(grid), 3]
    for x in range(3):
        Vx = np.clip(V + rng.uniform(-10.0, 10.0, N), grid[0], grid[-1])
        y[(x + 1) * N:(x + 2) * N] = table[np.rint((Vx - grid[0]) / 0.5).astype(int), x]
    post = np.repeat(np.arange(N, dtype=np.int64), np.diff(spec.row_ptr))
    net_of = np.searchsorted(spec.net_neuron_off, post, side="right") - 1
    pair = (spec.net_neuron_off[net_of].astype(np.int64) + spec.pre) * nt + spec.syn_type
    y[4 * N:4 * N + S] = rng.uniform(0.0, 0.8, N * nt).astype(np.float32)[pair]
    y[4 * N + S:] = rng.uniform(0.0, 0.5, N * nt).astype(np.float32)[pair]
    return y


def test_batched_as_benchmarked_single_step():
    from paper_1906_03958_gb300 import psst
    spec = ng.batched(n_nets=4096)
    N, S = spec.n_neurons, spec.n_synapses
    step0 = 2999  # inside many networks' pulse windows; (step0 + 1) is a multiple of the record stride
    y32 = _physiological_state(spec, 4242)
    with psst.Network(spec, rec_stride=10, rec_capacity=200) as net:
        net.autotune(200)
        net.set_graph_mode(True)
        net.set_state(y32)
        info = net.info()
        assert info["n_pair_gate_nets"] == spec.n_nets
        assert info["n_launch_classes"] > 1
        net.set_step(step0)
        net.integrate(1)
        net.status()
        got = net.get_state_numpy()
        frame = net.read_record()
    y64, _ = oracle.integrate(spec, y32.astype(np.float64), 1, step0=step0)
    err = step_error(got, y64, N, S)
    assert err <= 1e-5, err
    assert frame.shape == (1, N)
    np.testing.assert_array_equal(frame[0], got[:N])
