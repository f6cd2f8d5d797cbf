"""Helpers for the GPU parity tests."""
import numpy as np


def rel_err(got, ref):
    """Normwise max relative error max|g - o| / max|o|."""
    ref = np.asarray(ref, dtype=np.float64)
    d = np.abs(np.asarray(got, dtype=np.float64) - ref).max()
    s = np.abs(ref).max()
    return float(d / s) if s > 0 else float(d)


def cell_rel_err(got, ref, floor=1e-3):
    """Max over cells of |g - o| / |o| for cells with |o| >= floor * max|o|."""
    ref = np.asarray(ref, dtype=np.float64)
    got = np.asarray(got, dtype=np.float64)
    s = np.abs(ref).max()
    if s == 0:
        return float(np.abs(got).max())
    m = np.abs(ref) >= floor * s
    if not m.any():
        return 0.0
    return float((np.abs(got - ref)[m] / np.abs(ref)[m]).max())


# FP64 parity bar: max relative error against the FP64 oracle after the run's
# step count (the stated target is 1e-12; rounding differences between the
# GPU's fused multiply-adds and the oracle's separate roundings grow roughly
# linearly in the number of steps at a few ulps per step).
TOL_F64 = 1e-12


def f32_bound(steps):
    """A-priori bound for binary32 storage/arithmetic vs the FP64 oracle with
    values in [0, 1) and positive weights summing to 1: input rounding (2^-24),
    weight rounding (sum off by up to 5 * 2^-24 per step) and per-step
    rounding (up to 6 * 2^-24), accumulated linearly."""
    return (1 + 12 * max(steps, 1)) * 2.0 ** -24


def window_block(oracle, u0, w, steps, y0, y1, x0, x1, threads=None, box=False):
    """Oracle values of the cells [y0, y1) x [x0, x1) of u0 (array coordinates,
    ring included) after `steps` steps.  A cell's value after T steps depends
    only on the initial cells within distance T (also for the 3x3 box,
    box=True), so the oracle runs on the
    block plus a margin of T+1 cells (clipped at the array; the margin's edge is
    held constant, and its changes cannot reach the block within T steps)."""
    H, W = u0.shape
    r = steps + 1
    a0, a1 = max(0, y0 - r), min(H, y1 + r)
    b0, b1 = max(0, x0 - r), min(W, x1 + r)
    win = np.ascontiguousarray(u0[a0:a1, b0:b1])
    if threads is None:
        threads = oracle.max_threads()
    out = (oracle.box_run if box else oracle.run)(win, w, steps, threads=threads)
    return out[y0 - a0:y1 - a0, x0 - b0:x1 - b0]


def blocks_for(ny, nx, size=300):
    """Blocks (y0, y1, x0, x1) that cover the grid's corners (ring-adjacent
    cells, the first and last tiles), its middle and the middle of its left
    and bottom edges; each is `size` cells square (clipped), large enough to
    contain tile seams and CTA-group edges of every tile shape in both axes."""
    H, W = ny + 2, nx + 2
    s = min(size, H, W)
    cy, cx = (H - s) // 2, (W - s) // 2
    out = [(0, s, 0, s), (H - s, H, W - s, W), (cy, cy + s, cx, cx + s), (cy, cy + s, 0, s), (H - s, H, cx, cx + s)]
    seen, res = set(), []
    for b in out:
        if b not in seen:
            seen.add(b)
            res.append(b)
    return res
