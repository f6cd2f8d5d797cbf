"""The bounds-checked build (libj2d5pt_checked.so, J2D_BOUNDS_CHECK): every
shared-memory and global access of the blocked kernels is tested against its
buffer before it is made, and a failed test is reported as J2D_ERR_BOUNDS.
Every kernel family on tiny, thin and prime-sized grids, forward, adjoint,
batched and the 3x3 box, must report J2D_OK and agree with the oracle."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2306_03336_gb300 import j2d5pt, synth
from tests.gpu_util import TOL_F64, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def chk():
    import __graft_entry__
    __graft_entry__.build()
    return j2d5pt.load_checked()


def _status(lib, st):
    if st != j2d5pt.J2D_OK:
        raise j2d5pt.J2DError(st, lib.j2d5pt_last_error().decode())


def _run_checked(lib, u0, w, steps, algo, depth, wx, adjoint=False, box=False):
    import torch
    ny, nx = u0.shape[0] - 2, u0.shape[1] - 2
    h = ctypes.c_void_p()
    wa = np.ascontiguousarray(w, dtype=np.float64)
    plan = lib.j2d9pt_plan if box else lib.j2d5pt_plan
    _status(lib, plan(ctypes.byref(h), nx, ny, j2d5pt.J2D_F64, wa.ctypes.data_as(ctypes.c_void_p)))
    try:
        for opt, v in (("algo", j2d5pt.ALGO[algo]), ("depth", depth), ("tile_wx", wx)):
            _status(lib, lib.j2d5pt_set_option(h, j2d5pt.OPT[opt], v))
        pitch, off = ctypes.c_long(), ctypes.c_long()
        _status(lib, lib.j2d5pt_layout(h, 0, ctypes.byref(pitch), ctypes.byref(off)))
        src = torch.zeros((ny + 2, pitch.value), dtype=torch.float64, device="cuda")
        dst = torch.zeros_like(src)
        src[:, off.value:off.value + nx + 2] = torch.from_numpy(u0)
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        run = lib.j2d5pt_run_adjoint if adjoint else lib.j2d5pt_run
        _status(lib, run(h, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(dst.data_ptr()), steps, stream))
        _status(lib, lib.j2d5pt_sync_status(h))  # J2D_ERR_BOUNDS would raise here
        return dst[:, off.value:off.value + nx + 2].cpu().numpy()
    finally:
        lib.j2d5pt_plan_destroy(h)


SIZES = [(1, 1), (1, 7), (7, 1), (13, 17), (127, 131), (257, 300), (509, 3)]
FAMILIES = [("onestep", 0, 0), ("resident", 0, 0), ("bands", 3, 0), ("tiles", 3, 2), ("tiles", 5, 16), ("skewed", 3, 4),
            ("skewed", 6, 1), ("stream", 3, 0), ("stream", 6, 0)]


@pytest.mark.parametrize("algo,depth,wx", FAMILIES)
@pytest.mark.parametrize("nx,ny", SIZES)
def test_checked_forward(chk, algo, depth, wx, nx, ny):
    u0 = synth.field(nx, ny, 3000 + nx + ny)
    w = synth.weights(3001)
    for steps in (1, 7):
        got = _run_checked(chk, u0, w, steps, algo, depth, wx)
        assert rel_err(got, oracle.run(u0, w, steps)) <= TOL_F64, (algo, nx, ny, steps)


@pytest.mark.parametrize("algo,depth,wx", [("resident", 0, 0), ("bands", 3, 0), ("tiles", 3, 2)])
@pytest.mark.parametrize("nx,ny", [(1, 1), (13, 17), (257, 300)])
def test_checked_adjoint(chk, algo, depth, wx, nx, ny):
    lam = synth.field(nx, ny, 3100 + nx)
    w = synth.weights(3101)
    got = _run_checked(chk, lam, w, 5, algo, depth, wx, adjoint=True)
    assert rel_err(got, oracle.adjoint_run(lam, w, 5)) <= TOL_F64


@pytest.mark.parametrize("nx,ny", [(1, 1), (13, 17), (257, 300)])
@pytest.mark.parametrize("algo", ["onestep", "skewed"])
def test_checked_box(chk, nx, ny, algo):
    u0 = synth.field(nx, ny, 3200 + nx)
    w = synth.box_weights(3201)
    got = _run_checked(chk, u0, w, 6, algo, 3, 4, box=True)
    assert rel_err(got, oracle.box_run(u0, w, 6)) <= TOL_F64


def _run_checked_batch(lib, sizes, steps, algo, depth, wx, ctas):
    import torch
    n = len(sizes)
    nx = np.array([s[0] for s in sizes], dtype=np.int32)
    ny = np.array([s[1] for s in sizes], dtype=np.int32)
    w = np.stack([synth.weights(3300 + i) for i in range(n)])
    us = [synth.field(a, b, 3400 + i) for i, (a, b) in enumerate(sizes)]
    h = ctypes.c_void_p()
    _status(lib, lib.j2d5pt_plan_batched(ctypes.byref(h), n, nx.ctypes.data_as(ctypes.c_void_p),
                                         ny.ctypes.data_as(ctypes.c_void_p), j2d5pt.J2D_F64,
                                         np.ascontiguousarray(w).ctypes.data_as(ctypes.c_void_p)))
    try:
        for opt, v in (("algo", j2d5pt.ALGO[algo]), ("depth", depth), ("tile_wx", wx), ("ctas", ctas)):
            _status(lib, lib.j2d5pt_set_option(h, j2d5pt.OPT[opt], v))
        srcs, dsts, offs = [], [], []
        for i, ((a, b), u) in enumerate(zip(sizes, us)):
            pitch, off = ctypes.c_long(), ctypes.c_long()
            _status(lib, lib.j2d5pt_layout(h, i, ctypes.byref(pitch), ctypes.byref(off)))
            src = torch.zeros((b + 2, pitch.value), dtype=torch.float64, device="cuda")
            src[:, off.value:off.value + a + 2] = torch.from_numpy(u)
            srcs.append(src)
            dsts.append(torch.zeros_like(src))
            offs.append(off.value)
        pin = (ctypes.c_void_p * n)(*[t.data_ptr() for t in srcs])
        pout = (ctypes.c_void_p * n)(*[t.data_ptr() for t in dsts])
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        _status(lib, lib.j2d5pt_run_batched(h, ctypes.cast(pin, ctypes.c_void_p), ctypes.cast(pout, ctypes.c_void_p),
                                            steps, stream))
        _status(lib, lib.j2d5pt_sync_status(h))
        outs = [d[:, o:o + a + 2].cpu().numpy() for d, o, (a, _) in zip(dsts, offs, sizes)]
        return us, w, outs
    finally:
        lib.j2d5pt_plan_destroy(h)


@pytest.mark.parametrize("algo,depth,wx,ctas", [("tiles", 3, 2, 0), ("skewed", 3, 4, 0), ("resident", 0, 0, 0),
                                                ("resident", 0, 0, 2)])
def test_checked_batched(chk, algo, depth, wx, ctas):
    sizes = [(1, 1), (13, 17), (127, 31), (70, 3), (3, 70), (129, 40)]
    us, w, outs = _run_checked_batch(chk, sizes, 7, algo, depth, wx, ctas)
    for u, wi, got in zip(us, w, outs):
        assert rel_err(got, oracle.run(u, wi, 7)) <= TOL_F64, algo


@pytest.mark.parametrize("algo,depth,wx", [("tiles", 3, 2), ("bands", 3, 0), ("resident", 0, 0)])
@pytest.mark.parametrize("nx,ny", [(1, 1), (13, 17), (127, 131)])
def test_checked_states(chk, algo, depth, wx, nx, ny):
    """The state-keeping run's per-step stores through the checked build."""
    import torch
    u0 = synth.field(nx, ny, 3500 + nx)
    w = synth.weights(3501)
    steps = 6
    h = ctypes.c_void_p()
    wa = np.ascontiguousarray(w, dtype=np.float64)
    _status(chk, chk.j2d5pt_plan(ctypes.byref(h), nx, ny, j2d5pt.J2D_F64, wa.ctypes.data_as(ctypes.c_void_p)))
    try:
        for opt, v in (("algo", j2d5pt.ALGO[algo]), ("depth", depth), ("tile_wx", wx)):
            _status(chk, chk.j2d5pt_set_option(h, j2d5pt.OPT[opt], v))
        pitch, off = ctypes.c_long(), ctypes.c_long()
        _status(chk, chk.j2d5pt_layout(h, 0, ctypes.byref(pitch), ctypes.byref(off)))
        src = torch.zeros((ny + 2, pitch.value), dtype=torch.float64, device="cuda")
        src[:, off.value:off.value + nx + 2] = torch.from_numpy(u0)
        states = torch.zeros((steps, ny + 2, pitch.value), dtype=torch.float64, device="cuda")
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        _status(chk, chk.j2d5pt_run_states(h, ctypes.c_void_p(src.data_ptr()), ctypes.c_void_p(states.data_ptr()),
                                           steps, stream))
        _status(chk, chk.j2d5pt_sync_status(h))
        for t in range(steps):
            got = states[t, :, off.value:off.value + nx + 2].cpu().numpy()
            assert rel_err(got, oracle.run(u0, w, t + 1)) <= TOL_F64, (algo, t + 1)
    finally:
        chk.j2d5pt_plan_destroy(h)
