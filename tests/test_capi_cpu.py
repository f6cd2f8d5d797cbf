"""Host-side checks of the C ABI that need no GPU: the library loads, exports
every function include/j2d5pt.h declares, and rejects bad arguments before
touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2306_03336_gb300 import build as libbuild
from paper_2306_03336_gb300 import j2d5pt

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "j2d5pt.h")


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return j2d5pt.load()


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(j2d[59]pt_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ["j2d5pt_plan", "j2d5pt_run", "j2d5pt_plan_batched", "j2d5pt_run_batched",
                 "j2d5pt_run_adjoint", "j2d5pt_weight_grad", "j2d5pt_plan_destroy", "j2d5pt_last_error"]:
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_checked_build_exports_every_declared_symbol(lib):
    """The bounds-checked variant (J2D_BOUNDS_CHECK) is built beside the
    regular library and exposes the same C ABI."""
    chk = j2d5pt.load_checked()
    for name in declared_functions():
        assert hasattr(chk, name), name
    assert "bounds-checked" in chk.j2d5pt_version().decode()
    assert "bounds-checked" not in j2d5pt.j2d5pt_version()


def test_version_and_last_error(lib):
    assert "sm_103a" in j2d5pt.j2d5pt_version()
    assert isinstance(j2d5pt.j2d5pt_last_error(), str)


def test_argument_errors_before_device(lib):
    h = ctypes.c_void_p()
    w = np.array([0.2] * 5)
    wp = w.ctypes.data_as(ctypes.c_void_p)
    assert lib.j2d5pt_plan(ctypes.byref(h), 0, 5, 0, wp) == j2d5pt.J2D_ERR_ARG
    assert "nx=0" in j2d5pt.j2d5pt_last_error()
    assert lib.j2d5pt_plan(ctypes.byref(h), 5, -1, 0, wp) == j2d5pt.J2D_ERR_ARG
    assert lib.j2d5pt_plan(ctypes.byref(h), 5, 5, 7, wp) == j2d5pt.J2D_ERR_ARG
    assert lib.j2d5pt_plan(ctypes.byref(h), 5, 5, 0, None) == j2d5pt.J2D_ERR_ARG
    assert lib.j2d5pt_plan(None, 5, 5, 0, wp) == j2d5pt.J2D_ERR_ARG
    bad = np.array([0.2, np.nan, 0.2, 0.2, 0.2])
    assert lib.j2d5pt_plan(ctypes.byref(h), 5, 5, 0, bad.ctypes.data_as(ctypes.c_void_p)) == j2d5pt.J2D_ERR_ARG
    assert lib.j2d5pt_run(None, None, None, 1, None) == j2d5pt.J2D_ERR_ARG
    assert lib.j2d5pt_run_adjoint(None, None, None, 1, None) == j2d5pt.J2D_ERR_ARG
    assert lib.j2d5pt_weight_grad(None, None, None, None, None) == j2d5pt.J2D_ERR_ARG
    assert lib.j2d5pt_set_option(None, 0, 1) == j2d5pt.J2D_ERR_ARG
    assert lib.j2d5pt_plan_destroy(None) == j2d5pt.J2D_ERR_ARG
    assert lib.j2d5pt_sync_status(None) == j2d5pt.J2D_ERR_ARG
    r = ctypes.c_double()
    assert lib.j2d5pt_measure_fma_rate(9, ctypes.byref(r)) == j2d5pt.J2D_ERR_ARG
    assert lib.j2d5pt_adjoint_step_wgrad(None, None, None, None, None, None) == j2d5pt.J2D_ERR_ARG
    assert lib.j2d5pt_measure_exact_rate(None) == j2d5pt.J2D_ERR_ARG
    assert lib.j2d5pt_measure_smem_bandwidth(None) == j2d5pt.J2D_ERR_ARG
    assert lib.j2d5pt_get_option(None, 9, None) == j2d5pt.J2D_ERR_ARG


def test_arith_info_without_gpu(lib):
    """The FP64 cell-evaluation contract is a property of the library: half of
    the cells (rows with y mod 4 in {0, 1}) on the integer path, 11 guard bits."""
    m, g = ctypes.c_uint(), ctypes.c_int()
    assert lib.j2d5pt_arith_info(ctypes.byref(m), ctypes.byref(g)) == j2d5pt.J2D_OK
    assert m.value == 0x0F and g.value == 11
    assert lib.j2d5pt_arith_info(None, None) == j2d5pt.J2D_OK
    assert j2d5pt.j2d5pt_arith_info() == (0x0F, 11)


def test_plan_without_gpu_reports_device_error(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    w = np.array([0.2] * 5)
    st = lib.j2d5pt_plan(ctypes.byref(h), 8, 8, 0, w.ctypes.data_as(ctypes.c_void_p))
    assert st == j2d5pt.J2D_ERR_DEVICE
    assert h.value is None


def _header_enum(prefix):
    """name -> value of the header's enumerators that start with prefix."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(%s[A-Z0-9_]+)\s*=\s*(\d+)" % prefix, src)}


def test_binding_enums_match_the_header():
    """The binding passes algorithms, options and status codes by the
    header's values (it marshals names to the C enumerators)."""
    algos = _header_enum("J2D_ALGO_")
    assert {("J2D_ALGO_" + k.upper()): v for k, v in j2d5pt.ALGO.items()} == algos
    opts = _header_enum("J2D_OPT_")
    assert {("J2D_OPT_" + k.upper()): v for k, v in j2d5pt.OPT.items()} == opts
    for name, v in _header_enum("J2D_ERR_").items():
        assert getattr(j2d5pt, name) == v, name
    assert algos["J2D_ALGO_STREAM"] == 6
