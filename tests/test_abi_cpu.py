"""The C-ABI library builds, loads and exports every entry point of include/rcp.h (no GPU needed)."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1703_09074_gb300 import _lib
    if not os.path.exists(_lib.LIB_PATH):
        from paper_1703_09074_gb300 import build
        build.build()
    return _lib.load()


def header_functions():
    text = open(os.path.join(ROOT, "include", "rcp.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rcp_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_method_entry_points():
    names = header_functions()
    for required in ("rcp_plan", "rcp_sketch", "rcp_compress", "rcp_als", "rcp_project"):
        assert required in names


def test_every_header_symbol_is_exported_and_bound(lib):
    from paper_1703_09074_gb300 import _lib
    names = header_functions()
    assert names, "no declarations parsed"
    for name in names:
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, name


def test_invalid_configurations_are_rejected_before_any_device_work(lib):
    from paper_1703_09074_gb300._lib import RcpConfig, RCP_EINVAL

    def cfg(**kw):
        c = RcpConfig()
        c.ndim = 3
        for k, d in enumerate((10, 10, 10)):
            c.dims[k] = d
        c.rank, c.oversample, c.power_iters, c.max_iters, c.tol = 3, 2, 1, 10, 1e-8
        for k, v in kw.items():
            setattr(c, k, v)
        return c

    h = ctypes.c_void_p()
    for bad in (dict(ndim=1), dict(ndim=9), dict(rank=0), dict(rank=65), dict(oversample=-1),
                dict(power_iters=-1), dict(max_iters=0), dict(tol=-1.0), dict(in_dtype=7),
                dict(precision=9)):
        assert lib.rcp_plan(ctypes.byref(cfg(**bad)), None, ctypes.byref(h)) == RCP_EINVAL, bad
    c = cfg()
    c.dims[1] = 0
    assert lib.rcp_plan(ctypes.byref(c), None, ctypes.byref(h)) == RCP_EINVAL
    # l_n = min(R + p, I_n, J_n) < R is rejected
    c = cfg(rank=5)
    c.dims[0] = 4
    assert lib.rcp_plan(ctypes.byref(c), None, ctypes.byref(h)) == RCP_EINVAL
    assert lib.rcp_plan(None, None, ctypes.byref(h)) == RCP_EINVAL


def test_null_plan_handling(lib):
    from paper_1703_09074_gb300._lib import RCP_EINVAL
    assert lib.rcp_width(None, 1) == -1
    assert lib.rcp_plan_destroy(None) == 0
    assert lib.rcp_sketch(None, None, 1, None) == RCP_EINVAL
    assert lib.rcp_als(None, None, None, None) == RCP_EINVAL
    assert lib.rcp_status_str(0) == b"ok"
    assert lib.rcp_status_str(99) == b"unknown status"
    assert lib.rcp_test_normals(0, 0, 0, -1, 1, None, None, None, None) == RCP_EINVAL
    assert lib.rcp_test_arith(7, None, None, 1, None, None, None) == RCP_EINVAL
    assert lib.rcp_test_arith(0, None, None, -1, None, None, None) == RCP_EINVAL
    assert lib.rcp_test_arith(1, None, None, 4, None, None, None) == RCP_EINVAL
