"""The allocation-free entry point, psst_integrate_grid_noalloc.

It serves callers that cannot allocate device memory (a framework's pool
that must not be bypassed, a memory-capped process, code that only gets
buffers from its caller): they pass their own device arrays, and the
kernel's extra memory is a fixed array compiled into the library.  This
test drives it through the C interface on caller-owned torch buffers and
checks it against psst_integrate in grid mode on two calls in a row.  It
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
        row_ptr=keep["row_ptr"].data_ptr(), syn_code=keep["syn_code"].data_ptr(),
        weight=keep["weight"].data_ptr(), neuron_type=keep["neuron_type"].data_ptr(),
        neuron_params=keep["neuron_params"].data_ptr(), syn_params=keep["syn_params"].data_ptr(),
        i_const=keep["i_const"].data_ptr(), pulse_amp=keep["pulse_amp"].data_ptr(),
        pulse_on=int(spec.pulse_on[0]), pulse_off=int(spec.pulse_off[0]),
        noise_seed=int(spec.noise_seed), noise_thresh=int(spec.noise_thresh),
        noise_amp=float(spec.noise_amp), dt=float(spec.dt), state=state.data_ptr(),
        rec=rec.data_ptr(), rec_stride=10, rec_capacity=rec.shape[0], err=err.data_ptr())
    return dn, keep


def test_noalloc_matches_grid_mode_on_two_calls():
    import torch
    from paper_1906_03958_gb300 import psst
    spec = ng.sparse_large(seed=61, n_e=1600, n_i=400)
    spec.pulse_amp = np.full(spec.n_neurons, 2.0, np.float32)
    spec.pulse_on[:] = 40
    spec.pulse_off[:] = 220
    K = 3
    # the no-alloc call keeps one gate per synapse: compare with gate_mode 1
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
            ref.integrate(150)
            ref.status()
            psst.integrate_grid_noalloc(dn, 150 * call, 150)
            torch.cuda.synchronize()
            assert int(err.item()) == 0
            want = ref.get_state().cpu().numpy()
            got = state.cpu().numpy()
            np.testing.assert_array_equal(got, want)
            frames = ref.read_record()
            np.testing.assert_array_equal(rec[: len(frames)].cpu().numpy(), frames)
        assert np.ptp(got[: spec.n_neurons]) > 1.0  # the network did move


def test_noalloc_rejects_oversized_network():
    from paper_1906_03958_gb300 import psst
    dn = psst.DeviceNetwork(n_neurons=70000, n_synapses=0, n_syn_types=1, item_chunks=0,
                            row_ptr=1, syn_code=1, weight=1, neuron_type=1, neuron_params=1,
                            syn_params=1, i_const=1, dt=0.01, state=1, err=1)
    rc = psst.load().psst_integrate_grid_noalloc(C.byref(dn), 0, 10, None)
    assert rc == -7  # PSST_ERR_UNSUPPORTED: 70000 x 1 gate maps exceed the fixed array's limit
