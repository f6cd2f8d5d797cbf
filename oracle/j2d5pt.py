"""ctypes wrapper around the C oracle (``j2d5pt_oracle.c``).  Test infrastructure.

All arrays are dense numpy arrays of shape (ny+2, nx+2), row-major, ring
included; weights are the five values {W, E, S, C, N} of the paper's
Listing 1 (Section 3.1).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "j2d5pt_oracle.c")
_LIB = os.path.join(_HERE, "liboracle_j2d5pt.so")
_lib = None


def lib_path():
    return _LIB


def build(force=False):
    """Compile the oracle with gcc: -O2, OpenMP over rows, no FP contraction."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
           "-shared", "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        I = ctypes.c_int
        L = ctypes.c_long
        lib.oracle_j2d5pt_step.argtypes = [I, I, P, P, P]
        lib.oracle_j2d5pt_step.restype = None
        lib.oracle_j2d5pt_run.argtypes = [I, I, P, P, P, L, I]
        lib.oracle_j2d5pt_run.restype = I
        lib.oracle_j2d5pt_run_f32.argtypes = [I, I, P, P, P, L, I]
        lib.oracle_j2d5pt_run_f32.restype = I
        lib.oracle_j2d5pt_adjoint_step.argtypes = [I, I, P, P, P]
        lib.oracle_j2d5pt_adjoint_step.restype = None
        lib.oracle_j2d5pt_adjoint_run.argtypes = [I, I, P, P, P, L]
        lib.oracle_j2d5pt_adjoint_run.restype = I
        lib.oracle_j2d5pt_weight_grad.argtypes = [I, I, P, P, P]
        lib.oracle_j2d5pt_weight_grad.restype = None
        lib.oracle_j2d5pt_grad.argtypes = [I, I, P, P, P, L, P, P]
        lib.oracle_j2d5pt_grad.restype = I
        lib.oracle_dot.argtypes = [I, I, P, P]
        lib.oracle_dot.restype = ctypes.c_double
        lib.oracle_j2d9pt_step.argtypes = [I, I, P, P, P]
        lib.oracle_j2d9pt_step.restype = None
        lib.oracle_j2d9pt_run.argtypes = [I, I, P, P, P, L, I]
        lib.oracle_j2d9pt_run.restype = I
        lib.oracle_j2d9pt_run_f32.argtypes = [I, I, P, P, P, L, I]
        lib.oracle_j2d9pt_run_f32.restype = I
        lib.oracle_max_threads.argtypes = []
        lib.oracle_max_threads.restype = I
        _lib = lib
    return _lib


def _grid(a, dtype=np.float64):
    a = np.ascontiguousarray(a, dtype=dtype)
    if a.ndim != 2 or a.shape[0] < 3 or a.shape[1] < 3:
        raise ValueError("expected a (ny+2, nx+2) array with ny, nx >= 1")
    return a, a.shape[1] - 2, a.shape[0] - 2


def _w(w, dtype=np.float64):
    w = np.ascontiguousarray(w, dtype=dtype).reshape(-1)
    if w.size != 5:
        raise ValueError("weights must be the five values W, E, S, C, N")
    return w


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def max_threads():
    return int(_load().oracle_max_threads())


def step(u, w):
    """One forward step (Listing 1), ring held constant."""
    u, nx, ny = _grid(u)
    w = _w(w)
    out = np.empty_like(u)
    _load().oracle_j2d5pt_step(nx, ny, _p(w), _p(u), _p(out))
    return out


def run(u0, w, steps, threads=1):
    """``steps`` forward steps; ``threads`` OpenMP threads over rows."""
    u0, nx, ny = _grid(u0)
    w = _w(w)
    out = np.empty_like(u0)
    if _load().oracle_j2d5pt_run(nx, ny, _p(w), _p(u0), _p(out), int(steps), int(threads)):
        raise MemoryError("oracle run: allocation failed")
    return out


def run_f32(u0, w, steps, threads=1):
    """The same iteration in binary32 storage and arithmetic (weights rounded to float)."""
    u0, nx, ny = _grid(u0, np.float32)
    w = _w(w, np.float32)
    out = np.empty_like(u0)
    if _load().oracle_j2d5pt_run_f32(nx, ny, _p(w), _p(u0), _p(out), int(steps), int(threads)):
        raise MemoryError("oracle run_f32: allocation failed")
    return out


def adjoint_step(lam1, w):
    """One adjoint step lam = M^T lam1 (literal transpose of the forward step)."""
    lam1, nx, ny = _grid(lam1)
    w = _w(w)
    out = np.empty_like(lam1)
    _load().oracle_j2d5pt_adjoint_step(nx, ny, _p(w), _p(lam1), _p(out))
    return out


def adjoint_run(lamT, w, steps):
    lamT, nx, ny = _grid(lamT)
    w = _w(w)
    out = np.empty_like(lamT)
    if _load().oracle_j2d5pt_adjoint_run(nx, ny, _p(w), _p(lamT), _p(out), int(steps)):
        raise MemoryError("oracle adjoint_run: allocation failed")
    return out


def weight_grad(u, lam1, dw=None):
    """dw[d] + sum_i lam1[i] * u[nbr_d(i)] over interior i, d = W, E, S, C, N."""
    u, nx, ny = _grid(u)
    lam1, nx2, ny2 = _grid(lam1)
    if (nx, ny) != (nx2, ny2):
        raise ValueError("shape mismatch")
    acc = np.zeros(5) if dw is None else np.array(dw, dtype=np.float64).reshape(5).copy()
    _load().oracle_j2d5pt_weight_grad(nx, ny, _p(u), _p(lam1), _p(acc))
    return acc


def grad(u0, w, g, steps):
    """Gradient of L = <g, u_T> with respect to u0 and to the weights (full trajectory)."""
    u0, nx, ny = _grid(u0)
    g, nx2, ny2 = _grid(g)
    if (nx, ny) != (nx2, ny2):
        raise ValueError("shape mismatch")
    w = _w(w)
    lam0 = np.empty_like(u0)
    dw = np.zeros(5)
    if _load().oracle_j2d5pt_grad(nx, ny, _p(w), _p(u0), _p(g), int(steps), _p(lam0), _p(dw)):
        raise MemoryError("oracle grad: allocation failed")
    return lam0, dw


def dot(a, b):
    """Compensated <a, b> over all cells."""
    a, nx, ny = _grid(a)
    b, nx2, ny2 = _grid(b)
    if (nx, ny) != (nx2, ny2):
        raise ValueError("shape mismatch")
    return float(_load().oracle_dot(nx, ny, _p(a), _p(b)))


def loss(u, g):
    """L = <g, u>."""
    return dot(g, u)


# ---- j2d9pt: the nine-point box stencil --------------------------------------

def _w9(w, dtype=np.float64):
    w = np.ascontiguousarray(w, dtype=dtype).reshape(-1)
    if w.size != 9:
        raise ValueError("box weights must be nine values, rows y-1, y, y+1 and columns x-1, x, x+1")
    return w


def box_step(u, w):
    """One step of the 3x3 box stencil (weights row by row from the y-1 row,
    x-1 first), ring held constant."""
    u, nx, ny = _grid(u)
    w = _w9(w)
    out = np.empty_like(u)
    _load().oracle_j2d9pt_step(nx, ny, _p(w), _p(u), _p(out))
    return out


def box_run(u0, w, steps, threads=1):
    """``steps`` steps of the 3x3 box stencil."""
    u0, nx, ny = _grid(u0)
    w = _w9(w)
    out = np.empty_like(u0)
    if _load().oracle_j2d9pt_run(nx, ny, _p(w), _p(u0), _p(out), int(steps), int(threads)):
        raise MemoryError("oracle box_run: allocation failed")
    return out


def box_run_f32(u0, w, steps, threads=1):
    """The box iteration in binary32 storage and arithmetic (weights rounded to float)."""
    u0, nx, ny = _grid(u0, np.float32)
    w = _w9(w, np.float32)
    out = np.empty_like(u0)
    if _load().oracle_j2d9pt_run_f32(nx, ny, _p(w), _p(u0), _p(out), int(steps), int(threads)):
        raise MemoryError("oracle box_run_f32: allocation failed")
    return out
