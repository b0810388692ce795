"""Thin Python binding of the C interface in ``include/psst.h``.

Argument marshalling only: every step of the integration runs in the CUDA
library ``_build/libpsst.so``.  There is no CPU fallback; if the library is
missing or cannot load, every entry point raises.

PyTorch provides device memory and streams: ``get_state``/``read_record``
can write straight into CUDA tensors, and every call takes the current torch
stream unless another one is given.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

MODE_AUTO, MODE_CTA, MODE_GRID = 0, 1, 2
METHOD_RK4, METHOD_EULER, METHOD_TABLEAU = 0, 1, 2
OK = 0
ERRORS = {-1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "NONFINITE", -5: "TIMEOUT",
          -6: "STATE", -7: "UNSUPPORTED"}

EXPORTED = ("psst_create_network", "psst_integrate", "psst_status", "psst_get_state",
            "psst_set_state", "psst_set_step", "psst_read_record", "psst_query",
            "psst_destroy_network", "psst_error_string", "psst_last_error",
            "psst_set_barrier_timeout", "psst_integrate_grid_noalloc", "psst_set_weights",
            "psst_set_neuron_params", "psst_adjoint", "psst_record_checkpoints",
            "psst_set_graph_mode", "psst_autotune")


class PsstError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"psst error {code} ({ERRORS.get(code, '?')}): {msg}")
        self.code = code


class NetworkDesc(C.Structure):
    _fields_ = [("n_nets", C.c_int32), ("net_neuron_off", C.c_void_p),
                ("neuron_type", C.c_void_p), ("n_neuron_types", C.c_int32),
                ("neuron_params", C.c_void_p), ("row_ptr", C.c_void_p), ("pre", C.c_void_p),
                ("weight", C.c_void_p), ("syn_type", C.c_void_p), ("n_syn_types", C.c_int32),
                ("syn_params", C.c_void_p), ("i_const", C.c_void_p), ("pulse_amp", C.c_void_p),
                ("pulse_on", C.c_void_p), ("pulse_off", C.c_void_p),
                ("noise_seed", C.c_uint64), ("noise_thresh", C.c_uint32),
                ("noise_amp", C.c_float), ("dt", C.c_float), ("init_state", C.c_void_p),
                ("rec_stride", C.c_int32), ("rec_capacity", C.c_int64), ("mode", C.c_int32),
                ("block_threads", C.c_int32), ("item_chunks", C.c_int32), ("device", C.c_int32),
                ("gate_mode", C.c_int32), ("method", C.c_int32), ("min_cluster", C.c_int32),
                ("rk_stages", C.c_int32), ("rk_a", C.c_float * 3), ("rk_b", C.c_float * 4)]


class DeviceNetwork(C.Structure):
    """psst_device_network: one network in caller-owned device arrays."""
    _fields_ = [("n_neurons", C.c_int64), ("n_synapses", C.c_int64), ("n_syn_types", C.c_int32),
                ("item_chunks", C.c_int32), ("n_neuron_types", C.c_int32), ("row_ptr", C.c_void_p),
                ("syn_code", C.c_void_p),
                ("weight", C.c_void_p), ("neuron_type", C.c_void_p), ("neuron_params", C.c_void_p),
                ("syn_params", C.c_void_p), ("i_const", C.c_void_p), ("pulse_amp", C.c_void_p),
                ("pulse_on", C.c_int64), ("pulse_off", C.c_int64), ("noise_seed", C.c_uint64),
                ("noise_thresh", C.c_uint32), ("noise_amp", C.c_float), ("dt", C.c_float),
                ("state", C.c_void_p), ("rec", C.c_void_p), ("rec_stride", C.c_int32),
                ("rec_capacity", C.c_int64), ("err", C.c_void_p)]


class Info(C.Structure):
    _fields_ = [("n_nets", C.c_int32), ("n_neurons", C.c_int64), ("n_synapses", C.c_int64),
                ("steps_done", C.c_int64), ("rec_frames", C.c_int64), ("mode", C.c_int32),
                ("block_threads", C.c_int32), ("item_chunks", C.c_int32), ("grid_ctas", C.c_int32),
                ("smem_bytes", C.c_int32), ("n_single_cta_nets", C.c_int32),
                ("n_cluster_nets", C.c_int32), ("n_launch_classes", C.c_int32),
                ("kernel_launches", C.c_int32), ("n_pair_gate_nets", C.c_int32),
                ("n_independent_nets", C.c_int32), ("ck_start", C.c_int64), ("ck_steps", C.c_int64)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = False):
    """Load libpsst.so (raises if it is missing and not built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        if not os.path.exists(path):
            if not build_if_missing:
                raise RuntimeError(f"CUDA library {path} is not built; run __graft_entry__.build()")
            _build.build()
        lib = C.CDLL(path)
        P, I32, I64, SZ = C.c_void_p, C.c_int, C.c_int64, C.c_size_t
        lib.psst_create_network.argtypes = [C.POINTER(NetworkDesc), C.POINTER(Allocator), C.POINTER(P)]
        lib.psst_integrate.argtypes = [P, I64, P]
        lib.psst_status.argtypes = [P, P]
        lib.psst_get_state.argtypes = [P, P, SZ, I32, P]
        lib.psst_set_state.argtypes = [P, P, SZ, I32, P]
        lib.psst_set_step.argtypes = [P, I64]
        lib.psst_set_barrier_timeout.argtypes = [P, I64]
        lib.psst_set_weights.argtypes = [P, P, SZ, I32, P]
        lib.psst_set_neuron_params.argtypes = [P, P, SZ, I32, P]
        lib.psst_adjoint.argtypes = [P, I64, P, I64, C.c_int32, P, P, P, P]
        lib.psst_record_checkpoints.argtypes = [P, C.c_int32, I64]
        lib.psst_set_graph_mode.argtypes = [P, I32]
        lib.psst_autotune.argtypes = [P, I64, P]
        lib.psst_integrate_grid_noalloc.argtypes = [C.POINTER(DeviceNetwork), I64, I64, P]
        lib.psst_read_record.argtypes = [P, P, SZ, C.POINTER(C.c_int64), I32, P]
        lib.psst_query.argtypes = [P, C.POINTER(Info)]
        lib.psst_destroy_network.argtypes = [P]
        lib.psst_error_string.argtypes = [I32]
        lib.psst_error_string.restype = C.c_char_p
        lib.psst_last_error.restype = C.c_char_p
        for name in EXPORTED:
            if name not in ("psst_error_string", "psst_last_error"):
                getattr(lib, name).restype = I32
        _lib = lib
        return lib


def _check(rc: int):
    if rc != OK:
        raise PsstError(rc, load().psst_last_error().decode())


def _stream_handle(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def integrate_grid_noalloc(net: DeviceNetwork, step0: int, n_steps: int, stream=None):
    """psst_integrate_grid_noalloc: integrate a network held in the
    caller's device arrays without any device allocation."""
    rc = load().psst_integrate_grid_noalloc(C.byref(net), int(step0), int(n_steps), _stream_handle(stream))
    if rc != OK:
        raise PsstError(rc, "psst_integrate_grid_noalloc failed (see psst.h for the cases of this code)")


def _arr(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    """psst_allocator: device-memory provider of a handle."""
    _fields_ = [("alloc", _ALLOC_FN), ("free", _FREE_FN), ("ctx", C.c_void_p)]


class TorchAllocator:
    """Serves a handle's device memory from PyTorch's caching allocator
    (uint8 tensors kept alive until the library frees them)."""

    def __init__(self, device: int):
        self.device = device
        self.blocks = {}

        def _alloc(nbytes, ctx):
            import torch
            try:
                t = torch.empty(int(nbytes), dtype=torch.uint8, device=f"cuda:{self.device}")
            except RuntimeError:
                return None
            p = t.data_ptr()
            self.blocks[p] = t
            return p

        def _free(ptr, ctx):
            self.blocks.pop(ptr, None)

        self._alloc, self._free = _ALLOC_FN(_alloc), _FREE_FN(_free)
        self.struct = Allocator(self._alloc, self._free, None)


class Network:
    """A batch of networks resident on one GPU (``psst_create_network``).
    ``allocator="torch"`` takes the handle's device memory from PyTorch's
    caching allocator instead of cudaMalloc.  ``tableau=(a, b)`` integrates
    with that explicit Runge-Kutta map (METHOD_TABLEAU: a = the n - 1
    coefficients a_{s+1} of the stages' starts y + dt a_{s+1} k_s, b = the n
    weights; 1 <= n <= 4)."""

    def __init__(self, spec, init_state=None, rec_stride: int = 0, rec_capacity: int = 0,
                 mode: int = MODE_AUTO, block_threads: int = 0, item_chunks: int = 0,
                 device: int | None = None, gate_mode: int = 0, method: int = 0, allocator=None,
                 min_cluster: int = 0, tableau=None):
        lib = load()
        rk_stages, rk_a, rk_b = 0, [0.0] * 3, [0.0] * 4
        if tableau is not None:
            a, b = (list(np.atleast_1d(np.asarray(x, np.float64))) for x in tableau)
            if not 1 <= len(b) <= 4 or len(a) != len(b) - 1:
                raise ValueError("a tableau has 1..4 stages and n_stages - 1 coefficients a")
            method, rk_stages = METHOD_TABLEAU, len(b)
            rk_a[:len(a)], rk_b[:len(b)] = a, b
        keep = dict(
            off=_arr(spec.net_neuron_off, np.int32), nt=_arr(spec.neuron_type, np.int32),
            np_=_arr(spec.neuron_params, np.float32), rp=_arr(spec.row_ptr, np.int64),
            pre=_arr(spec.pre, np.int32), w=_arr(spec.weight, np.float32),
            st=_arr(spec.syn_type, np.int32), sp=_arr(spec.syn_params, np.float32),
            ic=_arr(spec.i_const, np.float32), pa=_arr(spec.pulse_amp, np.float32),
            pon=_arr(spec.pulse_on, np.int64), poff=_arr(spec.pulse_off, np.int64))
        if init_state is not None:
            keep["init"] = _arr(init_state, np.float32)
        ptr = lambda k: keep[k].ctypes.data if k in keep else None
        if device is None:
            import torch
            device = torch.cuda.current_device()
        d = NetworkDesc(
            n_nets=spec.n_nets, net_neuron_off=ptr("off"), neuron_type=ptr("nt"),
            n_neuron_types=keep["np_"].shape[0], neuron_params=ptr("np_"), row_ptr=ptr("rp"),
            pre=ptr("pre"), weight=ptr("w"), syn_type=ptr("st"),
            n_syn_types=keep["sp"].shape[0], syn_params=ptr("sp"), i_const=ptr("ic"),
            pulse_amp=ptr("pa"), pulse_on=ptr("pon"), pulse_off=ptr("poff"),
            noise_seed=int(spec.noise_seed), noise_thresh=int(spec.noise_thresh),
            noise_amp=float(spec.noise_amp), dt=float(spec.dt), init_state=ptr("init"),
            rec_stride=int(rec_stride), rec_capacity=int(rec_capacity), mode=int(mode),
            block_threads=int(block_threads), item_chunks=int(item_chunks), device=int(device),
            gate_mode=int(gate_mode), method=int(method), min_cluster=int(min_cluster), rk_stages=rk_stages,
            rk_a=(C.c_float * 3)(*rk_a), rk_b=(C.c_float * 4)(*rk_b))
        self._allocator = TorchAllocator(device) if allocator == "torch" else allocator
        if self._allocator is not None and not isinstance(self._allocator, TorchAllocator):
            raise ValueError("allocator must be None or 'torch'")
        h = C.c_void_p()
        _check(lib.psst_create_network(C.byref(d), C.byref(self._allocator.struct) if self._allocator else None,
                                       C.byref(h)))
        self._h = h
        self.device = device
        self.N = spec.n_neurons
        self.S = spec.n_synapses
        self.dim = 4 * self.N + 2 * self.S
        self.rec_stride = rec_stride
        self._cap = int(rec_capacity) if rec_stride > 0 else 0
        self.n_ntypes = keep["np_"].shape[0]
        self.recording_checkpoints = False
        # what the weight and neuron tables currently hold (the last source
        # written), and a counter bumped by every write: autograd.PsstTrace
        # uses both to run a backward against the tables of its own forward
        self._w_src, self._p_src = spec.weight, spec.neuron_params
        self.tables_version = 0

    def __del__(self):
        self.close()

    def close(self):
        h = getattr(self, "_h", None)
        if h:
            load().psst_destroy_network(h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- stepping
    def integrate(self, n_steps: int, stream=None):
        _check(load().psst_integrate(self._h, int(n_steps), _stream_handle(stream)))

    def status(self, stream=None):
        _check(load().psst_status(self._h, _stream_handle(stream)))

    def set_step(self, step: int):
        _check(load().psst_set_step(self._h, int(step)))

    def set_graph_mode(self, enable: bool = True):
        """Replay the integrate launch sequence through a captured CUDA graph."""
        _check(load().psst_set_graph_mode(self._h, int(bool(enable))))

    def autotune(self, trial_steps: int = 200, stream=None):
        """Pick each size class's CTA size by timed trials (results unchanged)."""
        _check(load().psst_autotune(self._h, int(trial_steps), _stream_handle(stream)))

    def set_barrier_timeout(self, ns: int):
        _check(load().psst_set_barrier_timeout(self._h, int(ns)))

    # -- state
    def get_state(self, out=None, stream=None):
        """State [V, m, h, n, r, s] into ``out`` (CUDA tensor or numpy array);
        default: a new float32 CUDA tensor."""
        import torch
        if out is None:
            out = torch.empty(self.dim, dtype=torch.float32, device=f"cuda:{self.device}")
        on_dev = isinstance(out, torch.Tensor) and out.is_cuda
        ptr = out.data_ptr() if isinstance(out, torch.Tensor) else out.ctypes.data
        n = out.numel() if isinstance(out, torch.Tensor) else out.size
        _check(load().psst_get_state(self._h, ptr, n, int(on_dev), _stream_handle(stream)))
        return out

    def get_state_numpy(self) -> np.ndarray:
        out = np.empty(self.dim, np.float32)
        return self.get_state(out)

    def set_state(self, x, stream=None):
        import torch
        if isinstance(x, torch.Tensor):
            x = x.contiguous()
            assert x.dtype == torch.float32
            on_dev, ptr, n = int(x.is_cuda), x.data_ptr(), x.numel()
        else:
            x = _arr(x, np.float32)
            on_dev, ptr, n = 0, x.ctypes.data, x.size
        _check(load().psst_set_state(self._h, ptr, n, on_dev, _stream_handle(stream)))

    def set_weights(self, w, stream=None):
        """Synaptic weights [S] from a float32 CUDA tensor or host array."""
        self._set_table(load().psst_set_weights, w, stream)
        self._w_src = w
        self.tables_version += 1

    def set_neuron_params(self, p, stream=None):
        """Neuron-type table [n_types, 9] from a float32 CUDA tensor or host array."""
        self._set_table(load().psst_set_neuron_params, p, stream)
        self._p_src = p
        self.tables_version += 1

    def tables_source(self):
        """(weights, neuron table) last written into the network: the
        objects given to set_weights / set_neuron_params, or the spec's."""
        return self._w_src, self._p_src

    def _set_table(self, fn, x, stream):
        import torch
        if isinstance(x, torch.Tensor):
            x = x.detach().contiguous()
            assert x.dtype == torch.float32
            _check(fn(self._h, x.data_ptr(), x.numel(), int(x.is_cuda), _stream_handle(stream)))
        else:
            x = _arr(x, np.float32)
            _check(fn(self._h, x.ctypes.data, x.size, 0, _stream_handle(stream)))

    def record_checkpoints(self, every: int, max_steps: int):
        """Have later integrate calls store checkpoints for adjoint(..., ckpt_every=0)."""
        _check(load().psst_record_checkpoints(self._h, int(every), int(max_steps)))
        self.recording_checkpoints = every > 0

    def adjoint(self, n_steps: int, dL_dV, ckpt_every: int = 1000, stream=None):
        """Gradients (dL/dw [S], dL/dparams [n_types, 9], dL/d(V,m,h,n)_0 [4, N])
        of L = sum(dL_dV * V(frames)) over the next n_steps steps; dL_dV is a
        float32 CUDA tensor [frames, N]."""
        import torch
        dev = f"cuda:{self.device}"
        dl = dL_dV.detach().to(device=dev, dtype=torch.float32).contiguous()
        gw = torch.empty(self.S, dtype=torch.float32, device=dev)
        gp = torch.empty((self.n_ntypes, 9), dtype=torch.float32, device=dev)
        gy = torch.empty((4, self.N), dtype=torch.float32, device=dev)
        _check(load().psst_adjoint(self._h, int(n_steps), dl.data_ptr() if dl.numel() else None,
                                   dl.shape[0] if dl.dim() == 2 else 0, int(ckpt_every), gw.data_ptr(),
                                   gp.data_ptr(), gy.data_ptr(), _stream_handle(stream)))
        return gw, gp, gy

    def read_record(self, out=None, stream=None):
        """Recorded V frames [frames, N], oldest first (numpy unless ``out``
        is a CUDA tensor)."""
        info = self.info()
        cap = min(info["rec_frames"], self._cap)
        if out is None:
            out = np.empty((max(cap, 0), self.N), np.float32)
        import torch
        on_dev = isinstance(out, torch.Tensor) and out.is_cuda
        ptr = out.data_ptr() if isinstance(out, torch.Tensor) else out.ctypes.data
        frames = out.shape[0]
        got = C.c_int64()
        _check(load().psst_read_record(self._h, ptr if frames else None, frames, C.byref(got),
                                       int(on_dev), _stream_handle(stream)))
        return out[: got.value]

    def info(self) -> dict:
        i = Info()
        _check(load().psst_query(self._h, C.byref(i)))
        return {k: getattr(i, k) for k, _ in Info._fields_}
