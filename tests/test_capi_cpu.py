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


def test_stream_geometry_covers_the_grid(lib):
    """The stream schedule's bands and runs (host arithmetic, no device):
    every interior cell is stored by exactly one (band, run) unit, each
    band's stored columns start on a 16-byte vector and lie at least G >= k
    columns inside the 32 vectors it evaluates, and runs are as tall as the
    minimum the schedule keeps (or the whole grid)."""
    rng = np.random.Generator(np.random.PCG64(2306034900))
    cases = [(16384, 16384, "f64", 2, 3648), (16384, 16384, "f32", 8, 1824), (1, 1, "f64", 4, 1),
             (8592, 8328, "f32", 12, 1520), (3, 700, "f32", 4, 4000), (700, 3, "f64", 6, 100)]
    for _ in range(60):
        dt = str(rng.choice(["f64", "f32"]))
        depth = int(rng.choice([2, 3, 4, 6] if dt == "f64" else [4, 6, 8, 10, 12]))
        cases.append((int(rng.integers(1, 20000)), int(rng.integers(1, 20000)), dt, depth, int(rng.integers(1, 5000))))
    for nx, ny, dt, depth, warps in cases:
        q = j2d5pt.j2d5pt_stream_geometry(nx, ny, dt, depth, warps)
        V = 2 if dt == "f64" else 4
        off = V - 1  # the plan layout's element offset of column 0
        assert q["depth"] == depth and q["G"] >= depth and q["G"] % V == 0
        assert q["vw"] == 32 * V - 2 * q["G"] > 0
        cols = np.zeros(nx + 2, dtype=np.int64)
        for b in range(q["bands"]):
            lo, hi = 1 + b * q["vw"], min(1 + (b + 1) * q["vw"], nx + 1)
            assert lo <= nx
            assert (off + lo) % V == 0  # the first stored vector is aligned
            cols[lo:hi] += 1
        assert (cols[1:nx + 1] == 1).all() and cols[0] == 0 and cols[nx + 1] == 0, (nx, dt, depth)
        rows = np.zeros(ny + 2, dtype=np.int64)
        for r in range(q["runs"]):
            lo, hi = 1 + r * q["H"], min(1 + (r + 1) * q["H"], ny + 1)
            assert lo <= ny
            rows[lo:hi] += 1
        assert (rows[1:ny + 1] == 1).all(), (ny, q)
        hmin = (32 if dt == "f64" else 16) * depth
        assert q["runs"] == 1 or q["H"] >= hmin or ny < hmin, (ny, q)
    # the box has its own depths; argument errors are refused before any device call
    assert j2d5pt.j2d5pt_stream_geometry(1000, 1000, "f32", 8, 100, shape=9)["G"] == 8
    for bad in [(0, 5, "f64", 2, 10, 5), (5, 5, "f64", 5, 10, 5), (5, 5, "f32", 2, 10, 5), (5, 5, "f64", 2, 0, 5),
                (5, 5, "f64", 6, 10, 9)]:
        with pytest.raises(j2d5pt.J2DError) as e:
            j2d5pt.j2d5pt_stream_geometry(*bad[:5], shape=bad[5])
        assert e.value.status == j2d5pt.J2D_ERR_ARG
