"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module only draws random numbers; it holds none of the stencil's
arithmetic.  Fields are (ny+2, nx+2) arrays (one-cell ring included) drawn
uniform in [0, 1) from numpy's PCG64; weights are five uniform [0, 1) draws
divided by their FP64 sum, in the order W, E, S, C, N.
"""
import numpy as np

SEED_BASE = 2306033360
WEIGHT_SEED_OFFSET = 1000


def rng(seed):
    return np.random.Generator(np.random.PCG64(int(seed)))


def field(nx, ny, seed, dtype=np.float64):
    """Uniform [0,1) field of shape (ny+2, nx+2), ring included; FP32 is the RNE cast."""
    a = rng(seed).random((ny + 2, nx + 2))
    return a.astype(dtype) if dtype != np.float64 else a


def weights(seed):
    """Five uniform [0,1) values divided by their FP64 sum (W, E, S, C, N)."""
    w = rng(seed).random(5)
    return w / w.sum()


def box_weights(seed):
    """Nine uniform [0,1) values divided by their FP64 sum: the 3x3 box
    weights, rows y-1, y, y+1, columns x-1, x, x+1."""
    w = rng(seed).random(9)
    return w / w.sum()


def dyadic_weights():
    """Weights that are exact binary fractions summing exactly to 1."""
    return np.array([1 / 8, 1 / 8, 1 / 4, 1 / 4, 1 / 4])


def dyadic_field(nx, ny, seed, bits=10):
    """Multiples of 2**-bits in [0, 1): exact in FP64 and FP32."""
    return rng(seed).integers(0, 2 ** bits, size=(ny + 2, nx + 2)).astype(np.float64) / 2 ** bits


def batch_sizes(count, seed, lo=64, hi=1024):
    """Per-grid (nx, ny), each side uniform in [lo, hi]."""
    r = rng(seed)
    nx = r.integers(lo, hi + 1, size=count)
    ny = r.integers(lo, hi + 1, size=count)
    return [(int(a), int(b)) for a, b in zip(nx, ny)]


def unit_cells(nx, ny, count, seed):
    """`count` distinct interior cells (y, x), uniform, 1-based with ring offset."""
    r = rng(seed)
    flat = r.choice(nx * ny, size=count, replace=False)
    return [(int(f // nx) + 1, int(f % nx) + 1) for f in flat]


# The five benchmark workloads: data seed SEED_BASE+i, weight seed +1000.
WORKLOADS = {
    "j2d5pt_f64_512x512_16": dict(nx=512, ny=512, steps=16, dtype="f64", index=0),
    "j2d5pt_f64_2048x1536_1000": dict(nx=2048, ny=1536, steps=1000, dtype="f64", index=1),
    "j2d5pt_f64_16384x16384_1000": dict(nx=16384, ny=16384, steps=1000, dtype="f64", index=1),
    "j2d5pt_f32_16384x16384_1000": dict(nx=16384, ny=16384, steps=1000, dtype="f32", index=2),
    "j2d5pt_f64_batch256_200": dict(count=256, lo=64, hi=1024, steps=200, dtype="f64", index=3),
    "j2d5pt_f64_4096x4096_500_adjoint": dict(nx=4096, ny=4096, steps=500, dtype="f64", index=4,
                                              checkpoint=50),
}


def data_seed(index):
    return SEED_BASE + index


def weight_seed(index):
    return SEED_BASE + index + WEIGHT_SEED_OFFSET
