"""GPU discrete adjoint (psst_adjoint, FP32) against the FP64 oracle's adjoint
and FP64 central finite differences; the torch.autograd bridge."""
import numpy as np
import pytest

import oracle
from paper_1906_03958_gb300 import netgen as ng
from tests.helpers import grad_error

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-3


def _spec(seed=3, sets=1):
    hidden, start = ng.differentiated(n_sets=sets, seed=seed, n_pn=12, n_ln=4)
    for s in (hidden, start):
        s.pulse_on[:] = 5
        s.pulse_off[:] = 10_000
    return hidden, start


def _gpu_adjoint(spec, nsteps, dLdV, stride, ckpt=50, step0=0):
    import torch
    from paper_1906_03958_gb300 import psst
    with psst.Network(spec, rec_stride=stride, rec_capacity=nsteps // stride + 1) as net:
        net.set_step(step0)
        gw, gp, gy = net.adjoint(nsteps, torch.from_numpy(dLdV.astype(np.float32)).cuda(), ckpt)
        net.status()
        return gw.cpu().numpy(), gp.cpu().numpy(), gy.cpu().numpy()


def test_adjoint_matches_oracle_adjoint():
    _, spec = _spec()
    rng = np.random.default_rng(0)
    nsteps, stride = 600, 10
    g = rng.standard_normal((nsteps // stride, spec.n_neurons))
    y0 = oracle.rest_state(spec)
    gy64, gw64, gp64 = oracle.adjoint(spec, y0, nsteps, g, stride, ckpt=100)
    gw, gp, gy = _gpu_adjoint(spec, nsteps, g, stride)
    assert grad_error(gw, gw64) <= GRAD_TOL
    assert grad_error(gp, gp64) <= GRAD_TOL
    N = spec.n_neurons
    assert grad_error(gy.ravel(), gy64[:4 * N]) <= GRAD_TOL


def test_adjoint_vs_fp64_finite_differences():
    # 10 random coordinates (weights and conductances), central differences
    # with h = 1e-6 max(1, |theta|) on the FP64 forward map
    _, spec = _spec(seed=4)
    net = oracle.OracleNet(spec)
    rng = np.random.default_rng(1)
    nsteps, stride = 500, 5
    g = rng.standard_normal((nsteps // stride, spec.n_neurons))
    y0 = oracle.rest_state(net)
    gw, gp, _ = _gpu_adjoint(spec, nsteps, g, stride)

    def loss():
        _, rec = oracle.integrate(net, y0, nsteps, rec_stride=stride)
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
        assert abs(got - want) <= GRAD_TOL * max(abs(want), 1e-2 * scale), (kind, idx, got, want)


def test_adjoint_batch_of_parameter_sets():
    _, spec = _spec(seed=5, sets=3)
    rng = np.random.default_rng(2)
    nsteps, stride = 300, 3
    g = rng.standard_normal((nsteps // stride, spec.n_neurons))
    gy64, gw64, gp64 = oracle.adjoint(spec, oracle.rest_state(spec), nsteps, g, stride, ckpt=64)
    gw, gp, _ = _gpu_adjoint(spec, nsteps, g, stride, ckpt=64)
    for b in range(spec.n_nets):
        s0, s1 = spec.row_ptr[spec.net_neuron_off[b]], spec.row_ptr[spec.net_neuron_off[b + 1]]
        assert grad_error(gw[s0:s1], gw64[s0:s1]) <= GRAD_TOL
        assert grad_error(gp[2 * b:2 * b + 2], gp64[2 * b:2 * b + 2]) <= GRAD_TOL


def test_checkpoint_spacing_and_step_offset():
    _, spec = _spec(seed=6)
    rng = np.random.default_rng(3)
    nsteps, stride, step0 = 240, 4, 2
    frames = (step0 + nsteps) // stride - step0 // stride
    g = rng.standard_normal((frames, spec.n_neurons))
    a = _gpu_adjoint(spec, nsteps, g, stride, ckpt=7, step0=step0)
    b = _gpu_adjoint(spec, nsteps, g, stride, ckpt=240, step0=step0)
    for x, y in zip(a, b):
        assert grad_error(x, y) <= 1e-5
    _, gw64, _ = oracle.adjoint(spec, oracle.rest_state(spec), nsteps, g, stride, step0=step0)
    assert grad_error(a[0], gw64) <= GRAD_TOL


def test_nonuniform_gates_are_rejected():
    from paper_1906_03958_gb300 import psst
    import torch
    _, spec = _spec(seed=7)
    y = oracle.rest_state(spec).astype(np.float32)
    N = spec.n_neurons
    y[4 * N + 3] = 0.5  # one gate differs from the other gates of its pair
    with psst.Network(spec, init_state=y, rec_stride=10, rec_capacity=10) as net:
        net.adjoint(50, torch.zeros((5, N), device="cuda"), 10)
        with pytest.raises(psst.PsstError) as ei:
            net.status()
        assert ei.value.code == -7


def test_autograd_mse_loss():
    import torch
    from paper_1906_03958_gb300 import psst
    from paper_1906_03958_gb300.autograd import trace
    hidden, start = _spec(seed=8)
    nsteps = 400
    N = hidden.n_neurons
    pn = torch.zeros(N, dtype=torch.bool, device="cuda")
    pn[:12] = True
    with psst.Network(hidden, rec_stride=1, rec_capacity=nsteps) as nh:
        target = trace(nh, torch.from_numpy(hidden.weight).cuda(), torch.from_numpy(hidden.neuron_params).cuda(),
                       nsteps).detach()
    with psst.Network(start, rec_stride=1, rec_capacity=nsteps) as net:
        w = torch.from_numpy(start.weight).cuda().requires_grad_(True)
        p = torch.from_numpy(start.neuron_params).cuda().requires_grad_(True)
        v = trace(net, w, p, nsteps)
        loss = ((v[:, pn] - target[:, pn]) ** 2).mean()
        loss.backward()
        assert net.info()["steps_done"] == nsteps
    dLdV = np.zeros((nsteps, N))
    diff = (v - target).detach().cpu().numpy()
    dLdV[:, :12] = 2.0 * diff[:, :12] / (nsteps * 12)
    _, gw64, gp64 = oracle.adjoint(start, oracle.rest_state(start), nsteps, dLdV, 1)
    assert grad_error(w.grad.cpu().numpy(), gw64) <= GRAD_TOL
    assert grad_error(p.grad.cpu().numpy(), gp64) <= GRAD_TOL
    assert float(loss.detach()) > 0


def test_recorded_checkpoints_match_own_checkpoints():
    import torch
    from paper_1906_03958_gb300 import psst
    _, spec = _spec(seed=9, sets=2)
    rng = np.random.default_rng(4)
    nsteps, stride, ck = 300, 5, 64
    g = torch.from_numpy(rng.standard_normal((nsteps // stride, spec.n_neurons)).astype(np.float32)).cuda()
    with psst.Network(spec, rec_stride=stride, rec_capacity=nsteps // stride) as net:
        own = net.adjoint(nsteps, g, ck)
        net.record_checkpoints(ck, nsteps)
        net.integrate(nsteps)
        rec = net.adjoint(nsteps, g, 0)
        net.status()
        for a, b in zip(own, rec):
            assert grad_error(b.cpu().numpy(), a.cpu().numpy()) <= 1e-5
        net.set_state(net.get_state())  # invalidates the recorded span
        with pytest.raises(psst.PsstError) as ei:
            net.adjoint(nsteps, g, 0)
        assert ei.value.code == -6


def test_autograd_with_recorded_checkpoints():
    import torch
    from paper_1906_03958_gb300 import psst
    from paper_1906_03958_gb300.autograd import trace
    _, spec = _spec(seed=10)
    nsteps = 200
    out = []
    for record in (False, True):
        with psst.Network(spec, rec_stride=2, rec_capacity=nsteps // 2) as net:
            if record:
                net.record_checkpoints(50, nsteps)
            w = torch.from_numpy(spec.weight).cuda().requires_grad_(True)
            p = torch.from_numpy(spec.neuron_params).cuda().requires_grad_(True)
            v = trace(net, w, p, nsteps, ckpt_every=50)
            (v ** 2).mean().backward()
            out.append((w.grad.cpu().numpy(), p.grad.cpu().numpy()))
    assert grad_error(out[1][0], out[0][0]) <= 1e-5
    assert grad_error(out[1][1], out[0][1]) <= 1e-5


def _with_duplicate_synapses(spec, seed=9):
    """The same network with a second synapse (own weight) for a random
    tenth of the existing ones: rows then hold two synapses of one
    (presynaptic neuron, type) pair."""
    rng = np.random.default_rng(seed)
    N = spec.n_neurons
    post = np.repeat(np.arange(N), np.diff(spec.row_ptr))
    dup = rng.random(spec.n_synapses) < 0.1
    post2 = np.concatenate([post, post[dup]])
    pre2 = np.concatenate([spec.pre, spec.pre[dup]])
    w2 = np.concatenate([spec.weight, rng.uniform(0.0, 0.2, int(dup.sum())).astype(np.float32)])
    t2 = np.concatenate([spec.syn_type, spec.syn_type[dup]])
    order = np.lexsort((t2, pre2, post2))
    row_ptr = np.zeros(N + 1, np.int64)
    np.add.at(row_ptr, post2 + 1, 1)
    return ng.NetworkSpec(
        net_neuron_off=spec.net_neuron_off, neuron_type=spec.neuron_type, neuron_params=spec.neuron_params,
        row_ptr=np.cumsum(row_ptr), pre=pre2[order].astype(np.int32), weight=w2[order].astype(np.float32),
        syn_type=t2[order].astype(np.int32), syn_params=spec.syn_params, i_const=spec.i_const,
        pulse_amp=spec.pulse_amp, pulse_on=spec.pulse_on, pulse_off=spec.pulse_off, dt=spec.dt,
        name=spec.name + "+duplicates")


def test_duplicate_synapses_forward_and_adjoint():
    # two synapses of one pair in a row: the forward's per-pair gates and the
    # adjoint's column sums (two slots of one column item from the same row)
    # against the oracle
    from paper_1906_03958_gb300 import psst
    from tests.helpers import step_error
    _, base = _spec(seed=11)
    spec = _with_duplicate_synapses(base)
    N, S = spec.n_neurons, spec.n_synapses
    assert S > base.n_synapses
    y32 = oracle.integrate(spec, oracle.rest_state(spec), 30)[0].astype(np.float32)
    y64, _ = oracle.integrate(spec, y32.astype(np.float64), 1, step0=30)
    with psst.Network(spec, init_state=y32) as net:
        assert net.info()["n_pair_gate_nets"] == 1
        net.set_step(30)
        net.integrate(1)
        net.status()
        assert step_error(net.get_state_numpy(), y64, N, S) <= 1e-5
    rng = np.random.default_rng(1)
    nsteps, stride = 300, 10
    g = rng.standard_normal((nsteps // stride, N))
    gy64, gw64, gp64 = oracle.adjoint(spec, oracle.rest_state(spec), nsteps, g, stride, ckpt=100)
    gw, gp, gy = _gpu_adjoint(spec, nsteps, g, stride)
    assert grad_error(gw, gw64) <= GRAD_TOL
    assert grad_error(gp, gp64) <= GRAD_TOL


def test_autograd_two_windows_before_one_backward():
    # Two trace windows of equal length with different weights, then one
    # backward of a loss over both: each window's gradient must be the
    # adjoint of its own span with its own tables (the network meanwhile
    # holds the second window's checkpoints and weights).  Reference: each
    # window's adjoint taken separately on a fresh network.
    import torch
    from paper_1906_03958_gb300 import psst
    from paper_1906_03958_gb300.autograd import trace
    _, spec = _spec(seed=12)
    nsteps, stride = 200, 2
    frames = nsteps // stride
    for record in (False, True):
        with psst.Network(spec, rec_stride=stride, rec_capacity=2 * frames) as net:
            if record:
                net.record_checkpoints(50, nsteps)
            w1 = torch.from_numpy(spec.weight).cuda().requires_grad_(True)
            p1 = torch.from_numpy(spec.neuron_params).cuda().requires_grad_(True)
            v1 = trace(net, w1, p1, nsteps, ckpt_every=50)
            y_mid = net.get_state().clone()
            w2 = (1.25 * w1.detach()).requires_grad_(True)
            p2 = p1.detach().clone().requires_grad_(True)
            v2 = trace(net, w2, p2, nsteps, ckpt_every=50)
            y_end = net.get_state().clone()
            ((v1 ** 2).mean() + (v2 ** 3).mean()).backward()
            # the network is left where the second window ended, with its tables
            assert net.info()["steps_done"] == 2 * nsteps
            assert torch.equal(net.get_state(), y_end)
        g1 = (2.0 * v1.detach() / v1.numel()).cpu().numpy()
        g2 = (3.0 * v2.detach() ** 2 / v2.numel()).cpu().numpy()
        spec2 = ng.NetworkSpec(**{k: getattr(spec, k) for k in spec.__dataclass_fields__})
        spec2.weight = (1.25 * spec.weight.astype(np.float32)).astype(np.float32)
        with psst.Network(spec, rec_stride=stride, rec_capacity=frames) as ref:
            r1 = ref.adjoint(nsteps, torch.from_numpy(g1).cuda(), 50)
        with psst.Network(spec2, init_state=y_mid.cpu().numpy(), rec_stride=stride,
                          rec_capacity=frames) as ref:
            ref.set_step(nsteps)
            r2 = ref.adjoint(nsteps, torch.from_numpy(g2).cuda(), 50)
            ref.status()
        assert grad_error(w1.grad.cpu().numpy(), r1[0].cpu().numpy()) <= 1e-5, record
        assert grad_error(p1.grad.cpu().numpy(), r1[1].cpu().numpy()) <= 1e-5, record
        assert grad_error(w2.grad.cpu().numpy(), r2[0].cpu().numpy()) <= 1e-5, record
        assert grad_error(p2.grad.cpu().numpy(), r2[1].cpu().numpy()) <= 1e-5, record


def test_adjoint_sparse_columns_against_oracle():
    # the antennal-lobe network (p = 0.5 per type pair, not dense): each
    # pair's column holds a random subset of rows, cut into several column
    # items of several chunks (rows dealt round-robin over the items), so the
    # sweep's gathers and item-order sums run on irregular columns
    spec = ng.antennal_lobe(seed=21)
    spec.pulse_on[:] = 5
    spec.pulse_off[:] = 10_000
    spec.pulse_amp[:] = np.where(spec.pulse_amp > 0, 8.0, 0.0)
    N = spec.n_neurons
    cnt = np.bincount(spec.pre * spec.syn_params.shape[0] + spec.syn_type)
    assert cnt.max() > 16 and np.count_nonzero((cnt > 0) & (cnt < N - 1)) > 0  # partial columns
    rng = np.random.default_rng(7)
    nsteps, stride = 300, 10
    g = rng.standard_normal((nsteps // stride, N))
    gy64, gw64, gp64 = oracle.adjoint(spec, oracle.rest_state(spec), nsteps, g, stride, ckpt=100)
    gw, gp, gy = _gpu_adjoint(spec, nsteps, g, stride, ckpt=100)
    assert grad_error(gw, gw64) <= GRAD_TOL, grad_error(gw, gw64)
    assert grad_error(gp, gp64) <= GRAD_TOL, grad_error(gp, gp64)
    assert grad_error(gy.ravel(), gy64[:4 * N]) <= GRAD_TOL
