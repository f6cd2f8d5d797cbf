"""Pins for the CPU oracle: facts fixed by the paper or by mathematics, none of
which re-types the oracle's own loops.

- golden impulse response (Section 3.1, Listing 1 orientation)
- exact agreement with a Kronecker-product matrix in rational arithmetic on
  dyadic inputs (brute force, exhaustive small sizes)
- rounding-error bound against exact rationals on random inputs
- closed-form separable eigenmodes of the forward and transposed operators
- invariants: constant field, linearity, ring constancy, maximum principle
- adjoint: dot-product identity and exact matrix transpose
- weight gradient: finite differences and Euler's identity for homogeneous maps
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


def _read_impulse():
    with open(os.path.join(GOLDEN, "impulse_listing1.txt")) as f:
        lines = [l.split() for l in f if l.strip() and not l.startswith("#")]
    hdr = lines[0]
    nx, ny, y0, x0 = int(hdr[1]), int(hdr[3]), int(hdr[5]), int(hdr[7])
    w = [float(v) for v in lines[1][1:]]
    cells = {(int(a), int(b)): float(c) for a, b, c in lines[2:]}
    return nx, ny, y0, x0, w, cells


def test_impulse_response_matches_listing1(oracle_mod):
    nx, ny, y0, x0, w, cells = _read_impulse()
    u = np.zeros((ny + 2, nx + 2))
    u[y0, x0] = 1.0
    out = oracle_mod.step(u, w)
    exp = np.zeros_like(u)
    for (y, x), v in cells.items():
        exp[y, x] = v
    assert np.array_equal(out, exp)


def test_impulse_weight_derivative_is_neighbour_value(oracle_mod):
    # d out[i] / d w_d = in[nbr_d(i)] (one step; Listing 1 read pattern)
    nx, ny = 5, 4
    u0 = synth.field(nx, ny, 7)
    w = synth.weights(8)
    y, x = 2, 3
    g = np.zeros_like(u0)
    g[y, x] = 1.0
    _, dw = oracle_mod.grad(u0, w, g, 1)
    exp = [u0[y, x - 1], u0[y, x + 1], u0[y - 1, x], u0[y, x], u0[y + 1, x]]
    assert np.array_equal(dw, np.array(exp))


@pytest.mark.parametrize("nx,ny", [(1, 1), (2, 3), (5, 4), (7, 7), (1, 6), (6, 1)])
def test_dyadic_exact_vs_rational_matrix(oracle_mod, nx, ny):
    w = synth.dyadic_weights()
    u0 = synth.dyadic_field(nx, ny, 11 + nx * 10 + ny)
    A = kron_ref.full_matrix(nx, ny, w, exact=True)
    v = kron_ref.to_fraction(u0)
    for steps in range(0, 9):
        out = oracle_mod.run(u0, w, steps)
        exact = np.array([[float(c) for c in row] for row in v])
        # every intermediate value is a dyadic rational with few bits: exact in FP64
        assert np.array_equal(out, exact), (nx, ny, steps)
        v = kron_ref.apply_steps(A, v, 1)


def test_exhaustive_small_sizes_dyadic(oracle_mod):
    w = synth.dyadic_weights()
    for nx in range(1, 10):
        for ny in range(1, 10):
            u0 = synth.dyadic_field(nx, ny, 1000 + 10 * nx + ny)
            A = kron_ref.full_matrix(nx, ny, w, exact=True)
            v = kron_ref.to_fraction(u0)
            for steps in range(0, 7):
                out = oracle_mod.run(u0, w, steps)
                exact = np.array([[float(c) for c in row] for row in v], dtype=np.float64)
                assert np.array_equal(out, exact), (nx, ny, steps)
                v = kron_ref.apply_steps(A, v, 1)


@pytest.mark.parametrize("nx,ny,steps", [(3, 2, 8), (5, 4, 6), (7, 7, 5)])
def test_rounding_bound_vs_exact_rationals(oracle_mod, nx, ny, steps):
    # seeded non-dyadic data: error <= steps * 6u * max|u0| (5-term sum, ||M||_inf ~ 1)
    w = synth.weights(21)
    u0 = synth.field(nx, ny, 22)
    A = kron_ref.full_matrix(nx, ny, [Fraction(float(x)) for x in w], exact=True)
    v = kron_ref.apply_steps(A, kron_ref.to_fraction(u0), steps)
    out = oracle_mod.run(u0, w, steps)
    err = max(abs(Fraction(float(o)) - e) for o, e in zip(out.reshape(-1), v.reshape(-1)))
    bound = steps * 6 * U * float(np.abs(u0).max())
    assert float(err) <= bound


@pytest.mark.parametrize("nx,ny", [(4, 3), (6, 6)])
def test_float_matrix_power(oracle_mod, nx, ny):
    # numpy matrix power of the Kronecker form (library routine) vs the oracle
    w = synth.weights(31)
    u0 = synth.field(nx, ny, 32)
    A = kron_ref.full_matrix(nx, ny, w)
    for steps in (1, 3, 10):
        ref = (np.linalg.matrix_power(A, steps) @ u0.reshape(-1)).reshape(u0.shape)
        out = oracle_mod.run(u0, w, steps)
        assert np.abs(out - ref).max() <= 2 * steps * 6 * U * np.abs(u0).max()


def _mode(nx, ny, w, p, q, transposed=False):
    W, E, S, C, N = w
    rx = math.sqrt(W / E) if not transposed else math.sqrt(E / W)
    ry = math.sqrt(S / N) if not transposed else math.sqrt(N / S)
    xs = np.arange(nx + 2)
    ys = np.arange(ny + 2)
    fx = rx ** xs * np.sin(p * math.pi * xs / (nx + 1))
    fy = ry ** ys * np.sin(q * math.pi * ys / (ny + 1))
    u = np.outer(fy, fx)
    u[0, :] = u[-1, :] = 0.0
    u[:, 0] = u[:, -1] = 0.0
    lam = C + 2 * math.sqrt(W * E) * math.cos(p * math.pi / (nx + 1)) \
        + 2 * math.sqrt(S * N) * math.cos(q * math.pi / (ny + 1))
    return u, lam


@pytest.mark.parametrize("nx,ny,p,q,steps", [(64, 48, 1, 1, 200), (33, 70, 2, 3, 50), (1, 9, 1, 1, 30)])
def test_separable_eigenmode_closed_form(oracle_mod, nx, ny, p, q, steps):
    # u0 = rx^x sin(p pi x/(nx+1)) ry^y sin(q pi y/(ny+1)), zero ring, rx = sqrt(W/E),
    # ry = sqrt(S/N): u_T = lambda^T u0 with lambda = C + 2 sqrt(WE) cos(.) + 2 sqrt(SN) cos(.)
    w = np.array([0.22, 0.18, 0.16, 0.24, 0.20])
    u0, lam = _mode(nx, ny, w, p, q)
    out = oracle_mod.run(u0, w, steps)
    ref = lam ** steps * u0
    scale = np.abs(u0).max()
    assert np.abs(out - ref).max() <= 64 * steps * U * scale
    # and the mode is not an eigenvector of the mirrored operator (orientation matters)
    wm = w[[1, 0, 4, 3, 2]]
    out_m = oracle_mod.run(u0, wm, steps)
    assert np.abs(out_m - ref).max() > 1e-6 * np.abs(ref).max()


def test_adjoint_eigenmode_closed_form(oracle_mod):
    nx, ny, steps = 40, 30, 60
    w = np.array([0.22, 0.18, 0.16, 0.24, 0.20])
    lamT, lam = _mode(nx, ny, w, 1, 2, transposed=True)
    out = oracle_mod.adjoint_run(lamT, w, steps)
    ref = lam ** steps * lamT
    assert np.abs(out[1:-1, 1:-1] - ref[1:-1, 1:-1]).max() <= 64 * steps * U * np.abs(lamT).max()


def test_constant_field_preserved(oracle_mod):
    nx, ny = 37, 23
    c = 0.6180339887
    u0 = np.full((ny + 2, nx + 2), c)
    out = oracle_mod.run(u0, synth.dyadic_weights(), 40)
    assert np.all(out == c)
    out = oracle_mod.run(u0, synth.weights(5), 40)
    assert np.abs(out - c).max() <= 40 * 6 * U * c


def test_linearity_exact_on_dyadic(oracle_mod):
    nx, ny = 13, 9
    w = synth.dyadic_weights()
    u = synth.dyadic_field(nx, ny, 1, bits=8)
    v = synth.dyadic_field(nx, ny, 2, bits=8)
    a, b = 0.75, -0.5
    lhs = oracle_mod.run(a * u + b * v, w, 5)
    rhs = a * oracle_mod.run(u, w, 5) + b * oracle_mod.run(v, w, 5)
    assert np.array_equal(lhs, rhs)


def test_ring_constant_and_max_principle_and_zero_steps(oracle_mod):
    nx, ny = 29, 31
    u0 = synth.field(nx, ny, 3)
    w = synth.weights(4)
    out = oracle_mod.run(u0, w, 25)
    for sl in (np.s_[0, :], np.s_[-1, :], np.s_[:, 0], np.s_[:, -1]):
        assert np.array_equal(out[sl], u0[sl])
    assert out.min() >= u0.min() - 1e-15 and out.max() <= u0.max() + 1e-15
    assert np.array_equal(oracle_mod.run(u0, w, 0), u0)


def test_threads_do_not_change_result(oracle_mod):
    u0 = synth.field(200, 150, 9)
    w = synth.weights(10)
    assert np.array_equal(oracle_mod.run(u0, w, 7, threads=1), oracle_mod.run(u0, w, 7, threads=4))


@pytest.mark.parametrize("steps", [1, 4])
def test_adjoint_dot_product_identity(oracle_mod, steps):
    nx, ny = 23, 17
    w = synth.weights(41)
    u = synth.field(nx, ny, 42)
    lam = synth.field(nx, ny, 43)
    lhs = oracle_mod.dot(oracle_mod.adjoint_run(lam, w, steps), u)
    rhs = oracle_mod.dot(lam, oracle_mod.run(u, w, steps))
    assert abs(lhs - rhs) <= 1e-13 * abs(rhs)


@pytest.mark.parametrize("nx,ny", [(1, 1), (3, 2), (4, 5)])
def test_adjoint_is_exact_matrix_transpose(oracle_mod, nx, ny):
    w = synth.dyadic_weights()
    lam = synth.dyadic_field(nx, ny, 51)
    A = kron_ref.full_matrix(nx, ny, w, exact=True)
    v = kron_ref.to_fraction(lam).reshape(-1)
    for steps in range(1, 5):
        v = A.T.dot(v)
        out = oracle_mod.adjoint_run(lam, w, steps)
        exact = np.array([float(c) for c in v]).reshape(lam.shape)
        assert np.array_equal(out, exact)


def test_weight_grad_vs_central_differences(oracle_mod):
    nx, ny, steps = 9, 7, 6
    u0 = synth.field(nx, ny, 61)
    g = synth.field(nx, ny, 62)
    w = synth.weights(63)
    _, dw = oracle_mod.grad(u0, w, g, steps)
    for d in range(5):
        h = 1e-5
        wp = w.copy(); wp[d] += h
        wm = w.copy(); wm[d] -= h
        fd = (oracle_mod.loss(oracle_mod.run(u0, wp, steps), g)
              - oracle_mod.loss(oracle_mod.run(u0, wm, steps), g)) / (2 * h)
        assert abs(fd - dw[d]) <= 1e-7 * abs(dw[d])


def test_weight_grad_euler_homogeneity(oracle_mod):
    # zero ring: u_T is homogeneous of degree T in w, so sum_d w_d dL/dw_d = T * L
    nx, ny, steps = 31, 27, 12
    u0 = synth.field(nx, ny, 71)
    u0[0, :] = u0[-1, :] = 0.0
    u0[:, 0] = u0[:, -1] = 0.0
    g = synth.field(nx, ny, 72)
    w = synth.weights(73)
    _, dw = oracle_mod.grad(u0, w, g, steps)
    L = oracle_mod.loss(oracle_mod.run(u0, w, steps), g)
    assert abs(float(np.dot(w, dw)) - steps * L) <= 1e-13 * abs(steps * L)


def test_grad_u0_is_transposed_power(oracle_mod):
    nx, ny, steps = 6, 5, 7
    w = synth.weights(81)
    u0 = synth.field(nx, ny, 82)
    g = synth.field(nx, ny, 83)
    lam0, _ = oracle_mod.grad(u0, w, g, steps)
    A = kron_ref.full_matrix(nx, ny, w)
    ref = (np.linalg.matrix_power(A.T, steps) @ g.reshape(-1)).reshape(g.shape)
    assert np.abs(lam0 - ref).max() <= 1e-14 * steps * np.abs(g).max() * 10


def test_dot_is_exactly_rounded_sum(oracle_mod):
    a = synth.field(50, 40, 91)
    b = synth.field(50, 40, 92)
    ref = math.fsum((a * b).reshape(-1).tolist())
    # products are rounded once each; compensated sum is within a few ulps of fsum
    assert abs(oracle_mod.dot(a, b) - ref) <= 4 * U * abs(ref)


def test_f32_oracle_exact_on_dyadic_and_bounded(oracle_mod):
    nx, ny = 21, 19
    w = synth.dyadic_weights()
    u0 = synth.dyadic_field(nx, ny, 101)
    for steps in range(0, 5):   # 10 + 3*steps bits <= 24: exact in binary32
        assert np.array_equal(oracle_mod.run_f32(u0, w, steps).astype(np.float64),
                              oracle_mod.run(u0, w, steps))
    w = synth.weights(102)
    u0 = synth.field(nx, ny, 103)
    steps = 50
    e = np.abs(oracle_mod.run_f32(u0, w, steps).astype(np.float64) - oracle_mod.run(u0, w, steps)).max()
    # input and weight rounding (2^-24 each) plus steps * 6 * 2^-24 per-step rounding
    assert e <= (steps * 6 + 2 + steps) * 2.0 ** -24
