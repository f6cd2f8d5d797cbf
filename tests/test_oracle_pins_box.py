"""Pins for the oracle of the second stencil shape, the 3x3 box (j2d9pt):
facts fixed by the definition or by mathematics, none of which re-types the
oracle's own loops.

- golden impulse response (tests/golden/impulse_box9.txt, derived by hand
  from the definition; orientation of Section 3.1, Listing 1)
- exact agreement with a Kronecker-product matrix in rational arithmetic on
  dyadic inputs (brute force, exhaustive small sizes)
- rounding-error bound against exact rationals on random inputs
- closed-form eigenmodes of a separable box (an outer product of two
  three-point weights), which fail for mirrored weights
- reduction to the j2d5pt oracle when the four corner weights are zero
- invariants: constant field, linearity, ring constancy, maximum principle
- the binary32 iteration: exact on dyadic inputs, within its bound otherwise
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2306_03336_gb300 import synth
from tests import kron_ref

U = 2.0 ** -53
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
# dyadic, asymmetric, summing exactly to 1
W_DYADIC = np.array([1, 1, 2, 2, 3, 2, 1, 3, 1], dtype=np.float64) / 16


def _read_golden():
    with open(os.path.join(GOLDEN, "impulse_box9.txt")) as f:
        lines = [l.split() for l in f if l.strip() and not l.startswith("#")]
    hdr = lines[0]
    nx, ny, y0, x0 = int(hdr[1]), int(hdr[3]), int(hdr[5]), int(hdr[7])
    w = [float(v) for v in lines[1][1:]]
    cells = {(int(a), int(b)): float(c) for a, b, c in lines[2:]}
    return nx, ny, y0, x0, w, cells


_box_weights = synth.box_weights


def test_box_impulse_golden(oracle_mod):
    nx, ny, y0, x0, w, cells = _read_golden()
    assert len(w) == 9 and len(cells) == 9
    u = np.zeros((ny + 2, nx + 2))
    u[y0, x0] = 1.0
    out = oracle_mod.box_step(u, w)
    exp = np.zeros_like(u)
    for (y, x), v in cells.items():
        exp[y, x] = v
    assert np.array_equal(out, exp)


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 3), (5, 4), (7, 7), (1, 6), (6, 1)])
def test_box_dyadic_exact_vs_rational_matrix(oracle_mod, nx, ny):
    u0 = synth.dyadic_field(nx, ny, 31 + nx * 10 + ny)
    A = kron_ref.full_matrix_box(nx, ny, W_DYADIC, exact=True)
    v = kron_ref.to_fraction(u0)
    for steps in range(0, 8):
        out = oracle_mod.box_run(u0, W_DYADIC, steps)
        exact = np.array([[float(c) for c in row] for row in v])
        assert np.array_equal(out, exact), (nx, ny, steps)
        v = kron_ref.apply_steps(A, v, 1)


def test_box_exhaustive_small_sizes_dyadic(oracle_mod):
    for nx in range(1, 8):
        for ny in range(1, 8):
            u0 = synth.dyadic_field(nx, ny, 2000 + 10 * nx + ny)
            A = kron_ref.full_matrix_box(nx, ny, W_DYADIC, exact=True)
            v = kron_ref.to_fraction(u0)
            for steps in range(0, 5):
                out = oracle_mod.box_run(u0, W_DYADIC, steps)
                exact = np.array([[float(c) for c in row] for row in v], dtype=np.float64)
                assert np.array_equal(out, exact), (nx, ny, steps)
                v = kron_ref.apply_steps(A, v, 1)


@pytest.mark.parametrize("nx,ny,steps", [(3, 2, 7), (5, 4, 5), (6, 6, 4)])
def test_box_rounding_bound_vs_exact_rationals(oracle_mod, nx, ny, steps):
    # seeded non-dyadic data and weights: a 9-term sum of non-negative terms
    # rounds at most 10 times per step, and ||M||_inf = 1
    w = _box_weights(41)
    u0 = synth.field(nx, ny, 42)
    A = kron_ref.full_matrix_box(nx, ny, [Fraction(float(x)) for x in w], exact=True)
    v = kron_ref.apply_steps(A, kron_ref.to_fraction(u0), steps)
    out = oracle_mod.box_run(u0, w, steps)
    err = max(abs(Fraction(float(o)) - e) for o, e in zip(out.reshape(-1), v.reshape(-1)))
    assert float(err) <= steps * 10 * U * float(np.abs(u0).max())


def _separable(p, q):
    return np.array([p[a] * q[b] for a in range(3) for b in range(3)])


def _mode(nx, ny, p, q, kx, ky):
    rx = math.sqrt(q[0] / q[2])
    ry = math.sqrt(p[0] / p[2])
    xs = np.arange(nx + 2)
    ys = np.arange(ny + 2)
    fx = rx ** xs * np.sin(kx * math.pi * xs / (nx + 1))
    fy = ry ** ys * np.sin(ky * math.pi * ys / (ny + 1))
    lam = (q[1] + 2 * math.sqrt(q[0] * q[2]) * math.cos(kx * math.pi / (nx + 1))) * \
          (p[1] + 2 * math.sqrt(p[0] * p[2]) * math.cos(ky * math.pi / (ny + 1)))
    u = np.outer(fy, fx)
    u[0, :] = u[-1, :] = 0.0
    u[:, 0] = u[:, -1] = 0.0
    return u, lam


@pytest.mark.parametrize("kx,ky", [(1, 1), (3, 2), (7, 5)])
def test_box_separable_eigenmode(oracle_mod, kx, ky):
    # w[dy][dx] = p[dy] q[dx]: the interior map is P_y kron Q_x, whose
    # tridiagonal factors have the eigenvectors r^i sin(k pi i / (n+1)),
    # r = sqrt(reads-below / reads-above); with a zero ring u_T = lam^T u_0
    nx, ny, steps = 30, 20, 8
    p, q = (0.3, 0.45, 0.25), (0.2, 0.5, 0.3)
    u0, lam = _mode(nx, ny, p, q, kx, ky)
    out = oracle_mod.box_run(u0, _separable(p, q), steps)
    exp = lam ** steps * u0
    assert np.abs(out - exp).max() <= 1e-12 * np.abs(exp).max()
    # the same mode is not an eigenvector of the mirrored weights (y-1 <-> y+1)
    out_m = oracle_mod.box_run(u0, _separable(p[::-1], q), steps)
    assert np.abs(out_m - exp).max() > 1e-6 * np.abs(exp).max()


def test_box_reduces_to_j2d5pt(oracle_mod):
    # corners zero: the box is the five-point stencil with W, E, S, C, N at
    # (y, x-1), (y, x+1), (y-1, x), (y, x), (y+1, x); on dyadic data both
    # oracles are exact, so they agree bit for bit
    W, E, S, C, N = 1 / 8, 1 / 8, 1 / 4, 1 / 4, 1 / 4
    box = np.array([0, S, 0, W, C, E, 0, N, 0])
    for nx, ny in ((9, 7), (1, 5), (13, 1)):
        u0 = synth.dyadic_field(nx, ny, 50 + nx)
        for steps in (1, 3, 6):
            assert np.array_equal(oracle_mod.box_run(u0, box, steps), oracle_mod.run(u0, [W, E, S, C, N], steps))


def test_box_invariants(oracle_mod):
    nx, ny, steps = 23, 17, 12
    w = _box_weights(61)
    # constant field (weights sum to 1 up to rounding): stays constant within the rounding bound
    c = 0.625
    u = np.full((ny + 2, nx + 2), c)
    out = oracle_mod.box_run(u, w, steps)
    assert np.abs(out - c).max() <= steps * 12 * U * c
    # exactly with dyadic weights
    assert np.array_equal(oracle_mod.box_run(u, W_DYADIC, steps), u)
    # linearity and ring constancy
    a = synth.field(nx, ny, 62)
    b = synth.field(nx, ny, 63)
    ra, rb = oracle_mod.box_run(a, w, steps), oracle_mod.box_run(b, w, steps)
    rab = oracle_mod.box_run(0.5 * a + 0.25 * b, w, steps)
    assert np.abs(rab - (0.5 * ra + 0.25 * rb)).max() <= 1e-14
    for sl in (np.s_[0, :], np.s_[-1, :], np.s_[:, 0], np.s_[:, -1]):
        assert np.array_equal(ra[sl], a[sl])
    # maximum principle: a convex combination stays inside [min, max] of the data
    assert ra.min() >= a.min() - 1e-15 and ra.max() <= a.max() + 1e-15


def test_box_f32(oracle_mod):
    nx, ny = 31, 19
    ud = synth.dyadic_field(nx, ny, 71)
    assert np.array_equal(oracle_mod.box_run_f32(ud, W_DYADIC, 3).astype(np.float64),
                          oracle_mod.box_run(ud, W_DYADIC, 3))
    u0 = synth.field(nx, ny, 72).astype(np.float32).astype(np.float64)
    w = _box_weights(73)
    steps = 20
    d = np.abs(oracle_mod.box_run_f32(u0, w, steps).astype(np.float64) - oracle_mod.box_run(u0, w, steps))
    assert d.max() <= (1 + 20 * steps) * 2.0 ** -24
