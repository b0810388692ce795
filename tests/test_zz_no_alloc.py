"""The allocation-free entry point, psst_integrate_grid_noalloc.

It serves callers that cannot allocate device memory (a framework's pool
that must not be bypassed, a memory-capped process, code that only gets
buffers from its caller): they pass their own device arrays, and the
kernel's extra memory is a fixed array compiled into the library.  This
test drives it through the C interface on caller-owned torch buffers and
checks it against psst_integrate in grid mode on two calls in a row (first-
and second-order synapses, a given and a chosen work-item size), and that
array contents out of range are refused before anything runs.  It
sits in a file of its own that pytest collects last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_1906_03958_gb300 import netgen as ng

pytestmark = pytest.mark.gpu


def _device_network(spec, state, rec, err, K):
    import torch
    from paper_1906_03958_gb300 import psst
    dev = state.device
    nt = spec.syn_params.shape[0]
    code = (spec.syn_type.astype(np.int64) << 24) | (spec.pre.astype(np.int64) * nt + spec.syn_type)
    keep = dict(
        row_ptr=torch.from_numpy(spec.row_ptr.astype(np.int64)).to(dev),
        syn_code=torch.from_numpy(code.astype(np.uint32).view(np.int32)).to(dev),
        weight=torch.from_numpy(spec.weight.astype(np.float32)).to(dev),
        neuron_type=torch.from_numpy(spec.neuron_type.astype(np.int32)).to(dev),
        neuron_params=torch.from_numpy(spec.neuron_params.astype(np.float32).ravel()).to(dev),
        syn_params=torch.from_numpy(spec.syn_params.astype(np.float32).ravel()).to(dev),
        i_const=torch.from_numpy(spec.i_const.astype(np.float32)).to(dev),
        pulse_amp=torch.from_numpy(spec.pulse_amp.astype(np.float32)).to(dev))
    dn = psst.DeviceNetwork(
        n_neurons=spec.n_neurons, n_synapses=spec.n_synapses, n_syn_types=nt, item_chunks=K,
        n_neuron_types=spec.neuron_params.shape[0],
        row_ptr=keep["row_ptr"].data_ptr(), syn_code=keep["syn_code"].data_ptr(),
        weight=keep["weight"].data_ptr(), neuron_type=keep["neuron_type"].data_ptr(),
        neuron_params=keep["neuron_params"].data_ptr(), syn_params=keep["syn_params"].data_ptr(),
        i_const=keep["i_const"].data_ptr(), pulse_amp=keep["pulse_amp"].data_ptr(),
        pulse_on=int(spec.pulse_on[0]), pulse_off=int(spec.pulse_off[0]),
        noise_seed=int(spec.noise_seed), noise_thresh=int(spec.noise_thresh),
        noise_amp=float(spec.noise_amp), dt=float(spec.dt), state=state.data_ptr(),
        rec=rec.data_ptr(), rec_stride=10, rec_capacity=rec.shape[0], err=err.data_ptr())
    return dn, keep


def _compare_two_calls(spec, K, steps=150):
    """Two no-alloc calls in a row against psst_integrate in grid mode with
    one gate per synapse and the same item_chunks (0: both choose)."""
    import torch
    from paper_1906_03958_gb300 import psst
    with psst.Network(spec, mode=psst.MODE_GRID, item_chunks=K, gate_mode=1, rec_stride=10,
                      rec_capacity=100) as ref:
        state = ref.get_state().clone()          # caller-owned buffers
        rec = torch.zeros((100, spec.n_neurons), dtype=torch.float32, device=state.device)
        err = torch.zeros(1, dtype=torch.int32, device=state.device)
        dn, keep = _device_network(spec, state, rec, err, K)
        for call in range(2):
            # the no-alloc call starts the remainders of its compensated step
            # sums at zero, as psst_integrate does after set_state
            ref.set_state(ref.get_state().clone())
            ref.integrate(steps)
            ref.status()
            psst.integrate_grid_noalloc(dn, steps * call, steps)
            torch.cuda.synchronize()
            assert int(err.item()) == 0
            want = ref.get_state().cpu().numpy()
            got = state.cpu().numpy()
            np.testing.assert_array_equal(got, want)
            frames = ref.read_record()
            np.testing.assert_array_equal(rec[: len(frames)].cpu().numpy(), frames)
        assert np.ptp(got[: spec.n_neurons]) > 1.0  # the network did move
        return ref.info()


def test_noalloc_matches_grid_mode_on_two_calls():
    spec = ng.sparse_large(seed=61, n_e=1600, n_i=400)
    spec.pulse_amp = np.full(spec.n_neurons, 2.0, np.float32)
    spec.pulse_on[:] = 40
    spec.pulse_off[:] = 220
    _compare_two_calls(spec, 3)


def test_noalloc_second_order_synapses():
    # the antennal lobe's LN -> PN GABA_B synapses are second order: the
    # plan's flag, the second table of maps and its scratch bound
    spec = ng.antennal_lobe(seed=62)
    spec.pulse_on[:] = 30
    assert (spec.syn_params[spec.syn_type, 0] != 0).any()
    _compare_two_calls(spec, 2)


def _hub_network(seed=63):
    """4000 HH neurons with pairs at p = 0.02 and neuron 0 receiving from
    every other neuron: the CTA that owns row 0 carries far more chunks than
    the average, so the work-item size follows the largest share."""
    rng = np.random.default_rng(seed)
    n = 4000
    post, pre = [], []
    for i in range(1, n):
        c = rng.choice(n - 1, size=rng.binomial(n - 1, 0.02), replace=False)
        c[c >= i] += 1
        post.append(np.full(c.size, i)), pre.append(c)
    post.append(np.zeros(n - 1, np.int64)), pre.append(np.arange(1, n))
    post, pre = np.concatenate(post), np.concatenate(pre)
    w = rng.lognormal(-2.0, 0.5, post.size)
    stype = (pre >= 3200).astype(np.int64)
    return ng.single_network(np.zeros(n), rng.uniform(0.0, 10.0, n), post, pre, w, stype,
                             ng.neuron_table(ng.HH), ng.synapse_table(ng.ACH, ng.GABA_A),
                             pulse_amp=np.full(n, 3.0), pulse_on=20, pulse_off=200, dt=ng.DT,
                             name="hub")


def test_noalloc_chooses_the_chunk_size_of_psst_integrate():
    spec = _hub_network()
    info = _compare_two_calls(spec, 0, steps=100)
    # row 0's CTA holds > 768 chunks, the average CTA about 160
    assert info["item_chunks"] == 2


@pytest.mark.parametrize("fault", ["row_ptr_end", "row_ptr_order", "syn_pre", "syn_type", "neuron_type"])
def test_noalloc_rejects_bad_array_contents(fault):
    import torch
    from paper_1906_03958_gb300 import psst
    spec = ng.antennal_lobe(seed=64)
    dev = torch.device("cuda", 0)
    nt = spec.syn_params.shape[0]
    state0 = torch.zeros(4 * spec.n_neurons + 2 * spec.n_synapses, dtype=torch.float32, device=dev)
    state0[: spec.n_neurons] = -60.0
    state = state0.clone()
    rec = torch.zeros((4, spec.n_neurons), dtype=torch.float32, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    dn, keep = _device_network(spec, state, rec, err, 2)
    # each case stays inside the arrays' extents: only the values are wrong
    if fault == "row_ptr_end":
        keep["row_ptr"][-1] -= 1
    elif fault == "row_ptr_order":
        keep["row_ptr"][5] = keep["row_ptr"][7] + 1
    elif fault == "syn_pre":
        keep["syn_code"][10] = (1 << 24) | (spec.n_neurons * nt + 1)
    elif fault == "syn_type":
        keep["syn_code"][11] = (5 << 24) | 5
    else:
        keep["neuron_type"][3] = spec.neuron_params.shape[0]
    torch.cuda.synchronize()
    rc = psst.load().psst_integrate_grid_noalloc(C.byref(dn), 0, 20, None)
    torch.cuda.synchronize()
    assert rc == -1  # PSST_ERR_INVALID_ARG
    assert int(err.item()) == 0
    assert torch.equal(state, state0)  # nothing integrated


def test_noalloc_rejects_oversized_network():
    from paper_1906_03958_gb300 import psst
    dn = psst.DeviceNetwork(n_neurons=70000, n_synapses=0, n_syn_types=1, item_chunks=0, n_neuron_types=1,
                            row_ptr=1, syn_code=1, weight=1, neuron_type=1, neuron_params=1,
                            syn_params=1, i_const=1, dt=0.01, state=1, err=1)
    rc = psst.load().psst_integrate_grid_noalloc(C.byref(dn), 0, 10, None)
    assert rc == -7  # PSST_ERR_UNSUPPORTED: 70000 x 1 gate maps exceed the fixed array's limit
