"""FP64 CPU oracle: test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``psst_oracle.c`` (plain C,
float64, built with gcc) through ctypes and shares no code with the CUDA
library: it reads the same seeded input arrays (any object with the
``NetworkSpec`` attributes) and widens them to float64.

Pinned functions and their pins live in ``tests/test_oracle_pins.py``,
``tests/test_oracle_adjoint.py`` and ``tests/test_oracle_tableau.py``.  The
Philox generator is pinned to its published known-answer vectors
(``tests/golden/philox_kat.json``) and to an independent library
implementation; its parity with the CUDA side is bit-exact by test.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "psst_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-std=c11"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (float64, no FMA contraction)."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


class _Net(C.Structure):
    _fields_ = [("N", C.c_int64), ("S", C.c_int64),
                ("ntype", C.c_void_p), ("nparams", C.c_void_p),
                ("row_ptr", C.c_void_p), ("pre", C.c_void_p), ("w", C.c_void_p),
                ("stype", C.c_void_p), ("sparams", C.c_void_p),
                ("i_const", C.c_void_p), ("pulse_amp", C.c_void_p),
                ("pulse_on", C.c_void_p), ("pulse_off", C.c_void_p),
                ("noise_seed", C.c_uint64), ("noise_thresh", C.c_uint32),
                ("noise_amp", C.c_double), ("dt", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            P = C.c_void_p
            _lib.orc_integrate.restype = C.c_int64
            _lib.orc_integrate.argtypes = [C.POINTER(_Net), P, C.c_int64, C.c_int64, C.c_int,
                                           C.c_int64, P, C.c_int64, P]
            _lib.orc_rhs.argtypes = [C.POINTER(_Net), P, P, P]
            _lib.orc_input.argtypes = [C.POINTER(_Net), C.c_int64, P]
            _lib.orc_linear_integrate.restype = C.c_int
            _lib.orc_linear_integrate.argtypes = [C.c_int64, P, P, C.c_double, C.c_int64, C.c_int, P]
            _lib.orc_philox4x32_10.argtypes = [P, P, P]
            _lib.orc_noise_event.restype = C.c_int
            _lib.orc_noise_event.argtypes = [C.c_uint64, C.c_uint32, C.c_int64, C.c_int64]
            _lib.orc_rates.argtypes = [C.c_double, P]
            _lib.orc_steady_gates.argtypes = [C.c_double, P]
            _lib.orc_vjp.argtypes = [C.POINTER(_Net), P, P, P, P, P]
            _lib.orc_linear_adjoint.restype = C.c_int
            _lib.orc_linear_adjoint.argtypes = [C.c_int64, P, P, C.c_double, C.c_int64, P, C.c_int, P]
            _lib.orc_adjoint.restype = C.c_int
            _lib.orc_adjoint.argtypes = [C.POINTER(_Net), P, C.c_int64, C.c_int64, C.c_int64, P, P, P, P,
                                         C.c_int64, C.c_int, P]
            _lib.orc_rates_deriv.argtypes = [C.c_double, P]
            _lib.orc_transmitter.restype = C.c_double
            _lib.orc_transmitter.argtypes = [C.c_double, C.c_double, C.c_double]
        return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _method(order: int, tableau):
    """(order, table) for the C entry points: order 4 (classic RK4) or 1
    (forward Euler), or with tableau = (a, b) the explicit Runge-Kutta map
    Y_1 = y, Y_s = y + h a[s-2] k_{s-1}, y' = y + h sum_s b[s-1] k_s
    (a: the n_stages - 1 coefficients a_{s,s-1}; b: the n_stages weights).
    The table array must outlive the call."""
    if tableau is None:
        if order not in (1, 4):
            raise ValueError("order must be 4 or 1 (or give a tableau)")
        return int(order), None
    a, b = (np.atleast_1d(np.asarray(x, np.float64)) for x in tableau)
    ns = len(b)
    if not 1 <= ns <= 4 or len(a) != ns - 1:
        raise ValueError("a tableau has 1..4 stages and n_stages - 1 coupling coefficients")
    tab = np.zeros(8, np.float64)
    tab[0] = ns
    tab[1:ns] = a
    tab[4:4 + ns] = b
    return 0, tab


def _tp(tab):
    return None if tab is None else _ptr(tab)


class OracleNet:
    """float64 copy of a network batch in the oracle's own layout."""

    def __init__(self, spec):
        noff = np.asarray(spec.net_neuron_off, np.int64)
        self.N = int(noff[-1])
        self.row_ptr = np.ascontiguousarray(spec.row_ptr, np.int64)
        self.S = int(self.row_ptr[-1])
        net_of_neuron = np.repeat(np.arange(len(noff) - 1), np.diff(noff))
        post = np.repeat(np.arange(self.N), np.diff(self.row_ptr))
        self.pre = (np.asarray(spec.pre, np.int64) + noff[net_of_neuron[post]]).astype(np.int64)
        self.w = np.asarray(spec.weight, np.float32).astype(np.float64)
        self.stype = np.ascontiguousarray(spec.syn_type, np.int32)
        self.sparams = np.asarray(spec.syn_params, np.float32).astype(np.float64).ravel()
        self.ntype = np.ascontiguousarray(spec.neuron_type, np.int32)
        self.nparams = np.asarray(spec.neuron_params, np.float32).astype(np.float64).ravel()
        self.i_const = np.asarray(spec.i_const, np.float32).astype(np.float64)
        self.pulse_amp = np.asarray(spec.pulse_amp, np.float32).astype(np.float64)
        self.pulse_on = np.asarray(spec.pulse_on, np.int64)[net_of_neuron].copy()
        self.pulse_off = np.asarray(spec.pulse_off, np.int64)[net_of_neuron].copy()
        self.c = _Net(self.N, self.S, _ptr(self.ntype), _ptr(self.nparams), _ptr(self.row_ptr),
                      _ptr(self.pre), _ptr(self.w), _ptr(self.stype), _ptr(self.sparams),
                      _ptr(self.i_const), _ptr(self.pulse_amp), _ptr(self.pulse_on),
                      _ptr(self.pulse_off), int(spec.noise_seed), int(spec.noise_thresh),
                      float(np.float32(spec.noise_amp)), float(np.float32(spec.dt)))
        self.dim = 4 * self.N + 2 * self.S


def as_net(spec_or_net) -> OracleNet:
    return spec_or_net if isinstance(spec_or_net, OracleNet) else OracleNet(spec_or_net)


def rest_state(spec, V0: float = -65.0) -> np.ndarray:
    """V = V0, gates at their steady state at V0, synaptic gates at 0."""
    net = as_net(spec)
    y = np.zeros(net.dim, np.float64)
    g = steady_gates(V0)
    y[: net.N] = V0
    for k in range(3):
        y[(k + 1) * net.N:(k + 2) * net.N] = g[k]
    return y


def integrate(spec, y0, nsteps: int, step0: int = 0, order: int = 4, rec_stride: int = 0, tableau=None):
    """Returns (y_final, rec[frames, N]).  order 4: RK4, 1: forward Euler;
    tableau = (a, b): that explicit Runge-Kutta map (see _method)."""
    order, tab = _method(order, tableau)
    net = as_net(spec)
    y = np.array(y0, np.float64, copy=True)
    assert y.shape == (net.dim,)
    cap = nsteps // rec_stride + 1 if rec_stride > 0 else 0
    rec = np.zeros((max(cap, 1), net.N), np.float64)
    got = lib().orc_integrate(C.byref(net.c), _ptr(y), int(step0), int(nsteps), order,
                              int(rec_stride), _ptr(rec), int(cap), _tp(tab))
    if got < 0:
        raise MemoryError("oracle integrate")
    return y, rec[:got]


def rhs(spec, y, step: int = 0) -> np.ndarray:
    net = as_net(spec)
    y = np.ascontiguousarray(y, np.float64)
    iext = input_current(net, step)
    dy = np.zeros(net.dim, np.float64)
    lib().orc_rhs(C.byref(net.c), _ptr(iext), _ptr(y), _ptr(dy))
    return dy


def input_current(spec, step: int) -> np.ndarray:
    net = as_net(spec)
    iext = np.zeros(net.N, np.float64)
    lib().orc_input(C.byref(net.c), int(step), _ptr(iext))
    return iext


def linear_integrate(A, y0, h: float, nsteps: int, order: int = 4, tableau=None) -> np.ndarray:
    order, tab = _method(order, tableau)
    A = np.ascontiguousarray(A, np.float64)
    y = np.array(y0, np.float64, copy=True)
    if lib().orc_linear_integrate(len(y), _ptr(A), _ptr(y), float(h), int(nsteps), order, _tp(tab)):
        raise MemoryError("oracle linear integrate")
    return y


class _Grads(C.Structure):
    _fields_ = [("gw", C.c_void_p), ("gnp", C.c_void_p)]


def vjp(spec, y, v, step: int = 0):
    """(J(y)^T v, dL/dw contribution, dL/dnparams contribution) at state y."""
    net = as_net(spec)
    y = np.ascontiguousarray(y, np.float64)
    v = np.ascontiguousarray(v, np.float64)
    iext = input_current(net, step)
    u = np.zeros(net.dim, np.float64)
    gw = np.zeros(net.S, np.float64)
    gnp = np.zeros(net.nparams.size, np.float64)
    g = _Grads(_ptr(gw), _ptr(gnp))
    lib().orc_vjp(C.byref(net.c), _ptr(iext), _ptr(y), _ptr(v), _ptr(u), C.addressof(g))
    return u, gw, gnp.reshape(-1, 9)


def linear_adjoint(A, y0, h: float, nsteps: int, lam_T, order: int = 4, tableau=None) -> np.ndarray:
    order, tab = _method(order, tableau)
    A = np.ascontiguousarray(A, np.float64)
    y0 = np.ascontiguousarray(y0, np.float64)
    lam = np.array(lam_T, np.float64, copy=True)
    if lib().orc_linear_adjoint(len(y0), _ptr(A), _ptr(y0), float(h), int(nsteps), _ptr(lam), order, _tp(tab)):
        raise MemoryError("oracle linear adjoint")
    return lam


def adjoint(spec, y0, nsteps: int, dLdV, rec_stride: int, step0: int = 0, ckpt: int = 100, order: int = 4,
            tableau=None):
    """Gradient of L = sum_f sum_i dLdV[f, i] V_i(frame f) over the RK4
    (order 4), Euler (order 1) or tableau trajectory; returns (dL/dy0,
    dL/dw, dL/dnparams[n_types, 9])."""
    order, tab = _method(order, tableau)
    net = as_net(spec)
    y0 = np.ascontiguousarray(y0, np.float64)
    dLdV = np.ascontiguousarray(dLdV, np.float64)
    gy = np.zeros(net.dim, np.float64)
    gw = np.zeros(net.S, np.float64)
    gnp = np.zeros(net.nparams.size, np.float64)
    if lib().orc_adjoint(C.byref(net.c), _ptr(y0), int(step0), int(nsteps), int(rec_stride), _ptr(dLdV),
                         _ptr(gy), _ptr(gw), _ptr(gnp), int(ckpt), order, _tp(tab)):
        raise MemoryError("oracle adjoint")
    return gy, gw, gnp.reshape(-1, 9)


def rates_deriv(V: float) -> np.ndarray:
    out = np.zeros(6, np.float64)
    lib().orc_rates_deriv(float(V), _ptr(out))
    return out


def philox(ctr, key) -> np.ndarray:
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def noise_event(seed: int, thresh: int, step: int, neuron: int) -> bool:
    return bool(lib().orc_noise_event(seed, thresh, step, neuron))


def rates(V: float) -> np.ndarray:
    out = np.zeros(6, np.float64)
    lib().orc_rates(float(V), _ptr(out))
    return out


def steady_gates(V: float) -> np.ndarray:
    out = np.zeros(3, np.float64)
    lib().orc_steady_gates(float(V), _ptr(out))
    return out


def transmitter(V: float, Vp: float, Kp: float) -> float:
    return lib().orc_transmitter(float(V), float(Vp), float(Kp))


def spike_times(rec: np.ndarray, dt_frame: float, t0: float = 0.0, theta: float = 0.0):
    """Upward crossings of theta per neuron, linearly interpolated between
    frames; rec[f] is the state at time t0 + (f+1) dt_frame."""
    rec = np.asarray(rec, np.float64)
    out = []
    for i in range(rec.shape[1]):
        v = rec[:, i]
        idx = np.nonzero((v[:-1] < theta) & (v[1:] >= theta))[0]
        frac = (theta - v[idx]) / (v[idx + 1] - v[idx])
        out.append(t0 + (idx + 1 + frac) * dt_frame)
    return out
