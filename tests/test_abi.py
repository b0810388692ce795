"""The C-ABI library loads, exports every declared symbol, and validates
descriptors on the host (no GPU compute)."""
import ctypes as C
import os
import re
import shutil
import subprocess

import numpy as np
import pytest

from paper_1906_03958_gb300 import build as pbuild
from paper_1906_03958_gb300 import netgen as ng
from paper_1906_03958_gb300 import psst

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_symbols():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(psst_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    if shutil.which("nvcc") is None and not os.path.exists(pbuild.LIB):
        pytest.skip("no nvcc to build the library")
    pbuild.build()
    return psst.load()


def test_every_declared_symbol_is_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 11
    out = subprocess.run(["nm", "-D", "--defined-only", pbuild.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (psst_\w+)", out))
    missing = [s for s in syms if s not in exported]
    assert not missing, missing
    for s in syms:
        assert getattr(lib, s) is not None
    assert set(psst.EXPORTED) <= set(syms)


def test_error_strings(lib):
    assert lib.psst_error_string(0) == b"ok"
    assert b"invalid" in lib.psst_error_string(-1)
    assert lib.psst_error_string(-99) == b"unknown error"


def _desc(spec, **kw):
    keep = {}

    def ptr(a, dt):
        a = np.ascontiguousarray(a, dt)
        keep[id(a)] = a
        return a.ctypes.data
    d = psst.NetworkDesc(
        n_nets=spec.n_nets, net_neuron_off=ptr(spec.net_neuron_off, np.int32),
        neuron_type=ptr(spec.neuron_type, np.int32), n_neuron_types=spec.neuron_params.shape[0],
        neuron_params=ptr(spec.neuron_params, np.float32), row_ptr=ptr(spec.row_ptr, np.int64),
        pre=ptr(spec.pre, np.int32), weight=ptr(spec.weight, np.float32),
        syn_type=ptr(spec.syn_type, np.int32), n_syn_types=spec.syn_params.shape[0],
        syn_params=ptr(spec.syn_params, np.float32), i_const=ptr(spec.i_const, np.float32),
        pulse_amp=None, pulse_on=None, pulse_off=None, dt=spec.dt, device=0)
    for k, v in kw.items():
        setattr(d, k, v)
    return d, keep


@pytest.mark.parametrize("field,value,needle", [
    ("n_nets", 0, b"n_nets"),
    ("dt", 0.0, b"dt"),
    ("n_syn_types", 9, b"n_syn_types"),
    ("noise_thresh", (1 << 24) + 1, b"noise_thresh"),
    ("block_threads", 100, b"block_threads"),
    ("item_chunks", 65, b"item_chunks"),
    ("rec_stride", -1, b"rec_stride"),
    ("gate_mode", 2, b"gate_mode"),
    ("method", 3, b"method"),
    ("mode", 3, b"mode"),
    ("min_cluster", 3, b"min_cluster"),
])
def test_invalid_descriptor_rejected_on_host(lib, field, value, needle):
    spec = ng.plain20()
    d, keep = _desc(spec, **{field: value})
    h = C.c_void_p()
    rc = lib.psst_create_network(C.byref(d), None, C.byref(h))
    assert rc == -1 and not h.value
    assert needle in lib.psst_last_error()


@pytest.mark.parametrize("kw,needle", [
    (dict(method=2, rk_stages=0), b"rk_stages"),
    (dict(method=2, rk_stages=5), b"rk_stages"),
    (dict(method=2, rk_stages=2, rk_b=(C.c_float * 4)(0.0, 0.0, 1.0, 1.0)), b"rk_b"),
    (dict(method=2, rk_stages=2, rk_a=(C.c_float * 3)(float("nan"), 0.0, 0.0),
          rk_b=(C.c_float * 4)(0.5, 0.5, 0.0, 0.0)), b"rk_a"),
])
def test_invalid_tableau_rejected_on_host(lib, kw, needle):
    d, keep = _desc(ng.plain20(), **kw)
    h = C.c_void_p()
    assert lib.psst_create_network(C.byref(d), None, C.byref(h)) == -1 and not h.value
    assert needle in lib.psst_last_error()


@pytest.mark.parametrize("tableau", [([0.5, 0.5], [0.5, 0.5]), ([], []), ([0.5] * 4, [0.2] * 5)])
def test_binding_rejects_malformed_tableau(lib, tableau):
    # a tableau has 1..4 weights b and one coefficient a fewer
    with pytest.raises(ValueError):
        psst.Network(ng.plain20(), tableau=tableau)


def test_out_of_range_presynaptic_index_rejected(lib):
    spec = ng.plain20()
    spec.pre = spec.pre.copy()
    spec.pre[5] = 20  # outside the 20-neuron network
    d, keep = _desc(spec)
    h = C.c_void_p()
    assert lib.psst_create_network(C.byref(d), None, C.byref(h)) == -1
    assert b"pre[5]" in lib.psst_last_error()


def test_null_handle_calls(lib):
    assert lib.psst_integrate(None, 1, None) == -1
    assert lib.psst_destroy_network(None) == 0
    assert lib.psst_query(None, None) == -1
