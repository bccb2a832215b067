"""CPU-side checks of the C ABI: the library loads, exports every function the header
declares, and its host-only entry points (status names, the parameter tuner, argument
validation that fails before any CUDA call) behave as documented.  No kernel runs here."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

from paper_1708_01135_gb300 import ewald as E

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "ewald.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(ewald_[a-z_]+)\s*\(", src)))


def _lib_or_skip():
    try:
        return E.lib()
    except RuntimeError as e:  # not built in this checkout
        pytest.skip(str(e))


def test_every_declared_function_is_exported():
    lib = _lib_or_skip()
    names = _header_functions()
    assert "ewald_create" in names and "ewald_submit" in names
    for name in names:
        assert hasattr(lib, name), name


def test_strerror_names_every_status():
    _lib_or_skip()
    for code in (0, 1, -1, -2, -3, -4, -5, -6, -7, -8, -9, -10):
        assert E.strerror(code).startswith("EWALD_")
    assert E.strerror(12345) == "EWALD_E_UNKNOWN"


def test_tune_rule_and_cutoff_choice():
    _lib_or_skip()
    # fixed r_c: beta = p / r_c, k_max = ceil(p beta L / pi), p = sqrt(-ln tol)
    rc, beta, km = E.tune(32768, 32.0, 1e-6, r_c=4.0)
    p = math.sqrt(-math.log(1e-6))
    assert rc == 4.0
    assert abs(beta - p / 4.0) < 1e-12
    assert km == math.ceil(p * beta * 32.0 / math.pi)
    # free r_c: a cutoff inside (0, L/2]
    rc, beta, km = E.tune(262144, 64.0, 1e-6)
    assert 0 < rc <= 32.0 and km >= 1


def test_tune_rejects_bad_arguments():
    _lib_or_skip()
    with pytest.raises(E.EwaldError):
        E.tune(1000, 10.0, 1e-6, r_c=6.0)   # r_c > L/2
    with pytest.raises(E.EwaldError):
        E.tune(1000, -1.0, 1e-6)


def test_create_rejects_bad_parameters_before_touching_the_device():
    lib = _lib_or_skip()
    h = ctypes.c_void_p()
    assert lib.ewald_create(8.0, 1.0, 4.5, 8, 0, ctypes.byref(h)) == E.E_CUTOFF
    assert lib.ewald_create(8.0, 1.0, 0.0, 8, 0, ctypes.byref(h)) == E.E_CUTOFF
    assert lib.ewald_create(-8.0, 1.0, 2.0, 8, 0, ctypes.byref(h)) == E.E_INVAL
    assert lib.ewald_create(8.0, 1.0, 2.0, 0, 0, ctypes.byref(h)) == E.E_INVAL
    assert lib.ewald_create(8.0, 1.0, 2.0, 200, 0, ctypes.byref(h)) == E.E_UNSUPPORTED
    assert lib.ewald_create(8.0, 1.0, 2.0, 8, 9, ctypes.byref(h)) == E.E_INVAL
    assert lib.ewald_create(8.0, float("nan"), 2.0, 8, 0, ctypes.byref(h)) == E.E_INVAL


def test_null_handles_are_rejected():
    lib = _lib_or_skip()
    e = (ctypes.c_double * 4)()
    assert lib.ewald_compute(None, 4, None, None, None, e, None) == E.E_INVAL
    assert lib.ewald_status_sync(None) == E.E_INVAL
    assert lib.ewald_server_destroy(None) == E.E_INVAL
    r = E._Result()
    assert lib.ewald_poll(None, 1, ctypes.byref(r)) == E.E_INVAL
    assert lib.ewald_md(None, 4, None, None, None, None, 1e-3, 10, None, None, None) == E.E_INVAL
    assert lib.ewald_set_spme(None, 32, 8) == E.E_INVAL
    assert lib.ewald_set_near_pairs(None, 1) == E.E_INVAL
    assert lib.ewald_set_lj(None, 1, None, None, None) == E.E_INVAL
    out = ctypes.c_double(0.0)
    assert lib.ewald_fma_peak(E.MIXED, ctypes.byref(out)) == E.E_INVAL   # FP32 or FP64 only
    assert lib.ewald_fma_peak(E.FP32, None) == E.E_INVAL


def test_realspace_erfc_fit_meets_its_bound():
    """The FP32 real-space kernels evaluate erfc(x) as t exp(-x^2) P(a t + b), t = 1 / (1 + p x),
    with the coefficients that csrc/fit_erfc.py derives.  Read them out of the kernel source
    and check the fit against scipy's double-precision erfc on [0, 8]: below 2e-8 relative in
    exact arithmetic, below 4e-7 with the kernel's FP32 rounding of t, u and Horner."""
    special = pytest.importorskip("scipy.special")
    src = open(os.path.join(ROOT, "paper_1708_01135_gb300", "csrc", "realspace.cu")).read()
    num = r"(-?[0-9]+\.[0-9]+(?:e-?[0-9]+)?)f"
    p = float(re.search(r"kErfcP = " + num, src).group(1))
    a = float(re.search(r"kErfcA = " + num, src).group(1))
    b = float(re.search(r"kErfcB = " + num, src).group(1))
    body = src[src.index("kErfcC[9] = {"):]
    body = body[:body.index("}")]
    coef = [float(v) for v in re.findall(num, body)]
    assert len(coef) == 9
    x = np.linspace(0.0, 8.0, 400001)
    t = 1.0 / (1.0 + p * x)
    u = a * t + b
    P = np.zeros_like(x)
    for c in reversed(coef):
        P = P * u + c
    ref = special.erfc(x)
    ok = ref > 1e-300
    exact = np.abs(t * np.exp(-x * x) * P / ref - 1)[ok]
    assert exact.max() < 2e-8, exact.max()
    x32 = x.astype(np.float32)
    t32 = (np.float32(1) / (np.float32(1) + np.float32(p) * x32)).astype(np.float32)
    u32 = (np.float32(a) * t32 + np.float32(b)).astype(np.float32)
    P32 = np.float32(coef[-1])
    for c in reversed(coef[:-1]):
        P32 = (P32 * u32 + np.float32(c)).astype(np.float32)
    f32 = np.abs(t32.astype(np.float64) * np.exp(-x * x) * P32.astype(np.float64) / ref - 1)[ok]
    assert f32.max() < 4e-7, f32.max()
