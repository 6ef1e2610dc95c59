"""CPU-side checks of the C ABI: the library builds, loads, exports every
entry point declared in include/fx.h, the ctypes signatures cover them, and
fx_create rejects bad parameters before touching the GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(fx_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1801_04834_gb300 import _abi, build
    build.build()
    return _abi.load()


def test_header_declares_entry_points():
    names = declared_functions()
    for n in ("fx_create", "fx_destroy", "fx_channelize", "fx_correct", "fx_correlate",
              "fx_last_error", "fx_query_sizes"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_covers_every_declared_symbol():
    from paper_1801_04834_gb300 import _abi
    assert set(declared_functions()) <= set(_abi.SIGNATURES)


def _params(**over):
    from paper_1801_04834_gb300 import _abi
    taps = np.ones(16 * 64, np.float32) / 1024
    centres = np.array([150e6])
    p = _abi.fx_params()
    p.n_stations, p.n_pols, p.n_subbands, p.n_channels, p.n_taps, p.n_spectra = 8, 2, 1, 64, 16, 32
    p.format, p.precision, p.sample_rate_hz, p.operand_scale, p.flags = 0, 0, 195312.5, 0.0, 0
    p.h_taps = taps.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    p.h_subband_centre_hz = centres.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    for k, v in over.items():
        setattr(p, k, v)
    return p, (taps, centres)


@pytest.mark.parametrize("field,value,status", [
    ("n_pols", 1, -5), ("n_channels", 32, -5), ("n_taps", 5, -5), ("n_stations", 0, -1),
    ("n_subbands", 0, -1), ("n_spectra", 0, -1), ("format", 7, -1), ("precision", 9, -1),
    ("sample_rate_hz", 0.0, -1), ("flags", 8, -1), ("max_coarse_shift", -1, -1), ("operand_scale", 3.0, -1),
])
def test_create_rejects_bad_params(lib, field, value, status):
    p, keep = _params(**{field: value})
    if field == "operand_scale":
        p.precision = 1
    h = ctypes.c_void_p(123)
    rc = lib.fx_create(ctypes.byref(p), ctypes.byref(h))
    assert rc == status
    assert h.value is None
    assert lib.fx_last_error().decode()


def test_create_rejects_null_pointers(lib):
    from paper_1801_04834_gb300 import _abi
    h = ctypes.c_void_p()
    assert lib.fx_create(None, ctypes.byref(h)) == -1
    p, keep = _params()
    p.h_taps = ctypes.POINTER(ctypes.c_float)()
    assert lib.fx_create(ctypes.byref(p), ctypes.byref(h)) == -1
    assert lib.fx_create(ctypes.byref(_params()[0]), None) == -1
    assert lib.fx_channelize(None, None, None, None) == -1
    assert lib.fx_correlate(None, None, None, None) == -1
    assert lib.fx_query_sizes(None, None) == -1
    lib.fx_destroy(None)
