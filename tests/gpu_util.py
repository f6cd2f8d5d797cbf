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
