"""The C-ABI library loads (no GPU needed) and exports every declared entry point."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    text = open(os.path.join(ROOT, "include", "nfl.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nfl_[A-Za-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1808_04580_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("nfl_plan_create", "nfl_degree", "nfl_apply_W", "nfl_apply_Ls",
                 "nfl_lanczos_k_smallest", "nfl_cg_solve", "nfl_plan_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_signatures_cover_the_header():
    from paper_1808_04580_gb300 import nfl
    assert sorted(nfl.SIGNATURES) == _declared()


def test_status_strings_without_gpu(lib):
    lib.nfl_status_string.restype = ctypes.c_char_p
    assert lib.nfl_status_string(0) == b"ok"
    assert b"degree" in lib.nfl_status_string(2)


def test_invalid_arguments_rejected_on_host(lib):
    """Argument checks run before any CUDA call, so they work without a GPU."""
    out = ctypes.c_void_p()
    fake = ctypes.c_void_p(16)
    f = lib.nfl_plan_create
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                  ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_void_p,
                  ctypes.POINTER(ctypes.c_void_p)]
    bad = [
        (fake, 0, 3, 0, 1.0, 32, 4, 4, -1.0, 0),     # n = 0
        (fake, 10, 4, 0, 1.0, 32, 4, 4, -1.0, 0),    # d = 4
        (fake, 10, 3, 5, 1.0, 32, 4, 4, -1.0, 0),    # unknown kernel
        (fake, 10, 3, -1, 1.0, 32, 4, 4, -1.0, 0),   # unknown kernel
        (fake, 10, 3, 0, -1.0, 32, 4, 4, -1.0, 0),   # sigma <= 0
        (fake, 10, 3, 0, 1.0, 30, 4, 4, -1.0, 0),    # N not a power of two
        (fake, 10, 3, 0, 1.0, 32, 0, 4, -1.0, 0),    # m = 0
        (fake, 10, 3, 0, 1.0, 32, 4, 4, 0.5, 0),     # eps_B >= 1/2
        (fake, 10, 3, 0, 1.0, 32, 4, 4, -1.0, 9),    # unknown precision
        (None, 10, 3, 0, 1.0, 32, 4, 4, -1.0, 0),    # null nodes
    ]
    for args in bad:
        assert f(*args, None, ctypes.byref(out)) == 1, args
        assert out.value is None


def test_host_products_reject_bad_arguments_without_gpu(lib):
    f = lib.nfl_apply_host
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_int64, ctypes.c_int]
    buf = (ctypes.c_double * 8)()
    assert f(None, 2, buf, 4, buf, 4, 1) == 1                      # no plan
    assert f(ctypes.c_void_p(16), 2, None, 4, buf, 4, 1) == 1      # no x
    assert f(ctypes.c_void_p(16), 3, buf, 4, buf, 4, 1) == 1       # unknown op
    assert f(ctypes.c_void_p(16), -1, buf, 4, buf, 4, 1) == 1      # unknown op
    assert f(ctypes.c_void_p(16), 2, buf, 4, buf, 4, 0) == 1       # no columns


def test_autotune_rejects_missing_plan_without_gpu(lib):
    f = lib.nfl_plan_autotune
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p]
    assert f(None, None) == 1
