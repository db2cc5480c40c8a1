"""The C ABI library builds for sm_103a, loads, and exports every declared symbol.

CPU-only: no call here touches a GPU (argument validation fails before any CUDA call).
"""
import ctypes
import os
import re

import pytest

from paper_2603_03019_gb300 import _build, hq

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(hq_\w+)\s*\(", text, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    return hq.load()


def test_header_declares_the_api():
    names = _declared_functions()
    for required in ("hq_create", "hq_load", "hq_solve", "hq_get_stationary", "hq_destroy",
                     "hq_get_utilisation", "hq_get_response_pattern", "hq_get_workload"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    raw = ctypes.CDLL(_build.LIB)
    missing = [n for n in _declared_functions() if not hasattr(raw, n)]
    assert not missing, missing


def test_library_is_built_for_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(_build.ARCH)
    assert os.path.exists(_build.LIB)


def test_invalid_arguments_rejected_without_gpu(lib):
    h = ctypes.c_void_p()
    assert lib.hq_create(0, 5, 0, 0, None, ctypes.byref(h)) == hq.HQ_EINVAL
    assert lib.hq_create(30, 5, 0, 0, None, ctypes.byref(h)) == hq.HQ_EINVAL
    assert lib.hq_create(8, 0, 0, 0, None, ctypes.byref(h)) == hq.HQ_EINVAL
    assert lib.hq_create(8, 5, 7, 0, None, ctypes.byref(h)) == hq.HQ_EINVAL
    assert lib.hq_create(8, 5, hq.HQ_FINITE, 0, None, ctypes.byref(h)) == hq.HQ_EINVAL
    assert b"finite buffer" in lib.hq_last_error()
    assert lib.hq_solve(None, None, None) == hq.HQ_EINVAL
    assert lib.hq_get_stationary(None, None, 0) == hq.HQ_EINVAL
    assert lib.hq_strerror(hq.HQ_EUNSTABLE).startswith(b"infinite queue")


def test_default_opts(lib):
    o = hq.hq_default_opts()
    assert o.tol == 1e-10 and o.tol_kind == hq.HQ_TOL_RESIDUAL
    assert o.precision == hq.HQ_PREC_FP32_DF64 and o.check_every >= 1
