"""Bit-exact check of the library's FP64 cell arithmetic on the GPU.

The oracle parity tests compare with a tolerance (1e-12), which would hide a
rare misrounding.  This test instead rebuilds, in exact rational arithmetic,
the two ways the kernels evaluate an FP64 cell (the contract stated for
j2d5pt_arith_info in include/j2d5pt.h) and requires every cell of every
algorithm to match bit for bit:

- the integer path: the correctly rounded (nearest-even) exact value of
  W*x[-1] + E*x[+1] + S*y[-1] + C*c + N*y[+1], for the cells the exact mask
  selects whose weights and values are positive normal, with product
  exponents within the guard and a normal result;
- otherwise the FMA chain S*ym, then fma with C, W, E, N in that order, each
  step rounded once.

Python's float(Fraction) is correctly rounded, so both are exact models.
Inputs are built to exercise rounding ties (short significands), the
exponent-spread fallback, zeros and negative values.
"""
from fractions import Fraction

import numpy as np
import pytest

from paper_2306_03336_gb300 import j2d5pt, synth

pytestmark = pytest.mark.gpu


def _biased_exp(v):
    return int((np.float64(v).view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF))


def _pos_normal(v):
    return v > 0 and 1 <= _biased_exp(v) <= 2046


def _rn(q):
    return float(q)  # correctly rounded: CPython divides big integers exactly


def model_cell(links, vals, x, y, mask, guard):
    """links and vals in the order (xm, xp, ym, c, yp)."""
    if (mask >> (((y & 3) << 1) | (x & 1))) & 1 and all(_pos_normal(w) for w in links) \
            and all(_pos_normal(v) for v in vals):
        E = [_biased_exp(w) + _biased_exp(v) for w, v in zip(links, vals)]
        if max(E) - min(E) <= guard:
            r = _rn(sum(Fraction(w) * Fraction(v) for w, v in zip(links, vals)))
            if 1 <= _biased_exp(r) <= 2046:
                return r
    F = Fraction
    r = _rn(F(links[2]) * F(vals[2]))
    for i in (3, 0, 1, 4):  # centre, x-1, x+1, y+1
        r = _rn(F(links[i]) * F(vals[i]) + F(r))
    return r


def model_step(u, w, mask, guard, adjoint=False):
    """One forward step (adjoint: interior cells away from the ring only)."""
    ny, nx = u.shape[0] - 2, u.shape[1] - 2
    W, E, S, C, N = (float(a) for a in w)
    links = (E, W, N, C, S) if adjoint else (W, E, S, C, N)
    out = u.copy()
    lo, hi_y, hi_x = (2, ny - 1, nx - 1) if adjoint else (1, ny, nx)
    for y in range(lo, hi_y + 1):
        for x in range(lo, hi_x + 1):
            vals = (u[y, x - 1], u[y, x + 1], u[y - 1, x], u[y, x], u[y + 1, x])
            out[y, x] = model_cell(links, [float(v) for v in vals], x, y, mask, guard)
    return out


def _short_significands(shape, rng, kmax=30, emin=-6):
    k = rng.integers(1, kmax + 1, size=shape)
    frac = np.floor(rng.random(shape) * 2.0 ** k) / 2.0 ** k
    return (1.0 + frac) * 2.0 ** rng.integers(emin, 1, size=shape) / 2


def _fields(nx, ny):
    rng = np.random.Generator(np.random.PCG64(2306033399))
    shape = (ny + 2, nx + 2)
    uni = synth.field(nx, ny, synth.data_seed(0))
    short = _short_significands(shape, rng)
    spread = synth.field(nx, ny, synth.data_seed(5)) * 2.0 ** -rng.integers(0, 40, size=shape)
    mixed = synth.field(nx, ny, synth.data_seed(6)) - 0.25
    mixed[rng.random(shape) < 0.05] = 0.0
    return {"uniform": uni, "short": short, "spread": spread, "mixed": mixed}


def _weights():
    rng = np.random.Generator(np.random.PCG64(2306033398))
    short = _short_significands(5, rng, kmax=26, emin=-3)
    return {"seeded": synth.weights(synth.weight_seed(1)), "short": short,
            "negative": np.array([0.3, -0.05, 0.25, 0.3, 0.2])}


NX, NY = 70, 45
ALGOS = ["onestep", "resident", "bands", "tiles", "skewed", "stream"]


@pytest.fixture(scope="module")
def arith():
    return j2d5pt.j2d5pt_arith_info()


@pytest.mark.parametrize("int_path", [1, 0])
@pytest.mark.parametrize("wname", ["seeded", "short", "negative"])
@pytest.mark.parametrize("fname", ["uniform", "short", "spread", "mixed"])
def test_cells_bit_exact(arith, fname, wname, int_path):
    mask, guard = arith
    mask = mask if int_path else 0
    u0 = _fields(NX, NY)[fname]
    w = _weights()[wname]
    steps = 3
    ref = u0
    for _ in range(steps):
        ref = model_step(ref, w, mask, guard)
    for algo in ALGOS:
        plan = j2d5pt.Plan(NX, NY, "f64", w).set("algo", algo).set("int_path", int_path)
        assert plan.get("int_path") == int_path
        if algo != "onestep":
            plan.set("depth", steps)
        src, dst = plan.to_device(u0), plan.empty()
        plan.run(src, dst, steps)
        plan.sync()
        got = plan.to_host(dst)
        plan.close()
        bad = np.argwhere(got != ref)
        assert bad.size == 0, "%s/%s/%s/int_path=%d: %d cells differ, first (y, x) = %s: %r vs model %r" % (
            algo, fname, wname, int_path, len(bad), tuple(bad[0]), got[tuple(bad[0])], ref[tuple(bad[0])])


def test_adjoint_interior_bit_exact(arith):
    mask, guard = arith
    u0 = _fields(NX, NY)["short"]
    w = _weights()["seeded"]
    ref = model_step(u0, w, mask, guard, adjoint=True)
    for algo in ALGOS:
        plan = j2d5pt.Plan(NX, NY, "f64", w).set("algo", algo)
        src, dst = plan.to_device(u0), plan.empty()
        plan.run_adjoint(src, dst, 1)
        plan.sync()
        got = plan.to_host(dst)
        plan.close()
        sl = np.s_[2:NY, 2:NX]
        bad = np.argwhere(got[sl] != ref[sl])
        assert bad.size == 0, "%s adjoint: %d cells differ" % (algo, len(bad))


def test_integer_path_is_used(arith):
    """The seeded uniform workload takes the integer path on the masked cells:
    there the result is the correctly rounded exact sum, which differs from
    the FMA chain on a sizeable share of cells."""
    mask, guard = arith
    assert mask != 0
    u0 = _fields(NX, NY)["uniform"]
    w = _weights()["seeded"]
    ref = model_step(u0, w, mask, guard)
    chain = model_step(u0, w, 0, guard)
    assert np.count_nonzero(ref != chain) > 0.05 * NX * NY * bin(mask).count("1") / 8
