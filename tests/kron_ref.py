"""Independent matrix form of one j2d5pt step, for pinning the oracle.

The full map over the (ny+2)(nx+2) cells is assembled from one-dimensional
shift matrices with Kronecker products (row-major, x fastest), not from the
oracle's loops: the interior block is
    C*I + W*(P_I kron Dx-) + E*(P_I kron Dx+) + S*(Dy- kron P_I) + N*(Dy+ kron P_I)
restricted to interior rows, where Dx- reads the x-1 neighbour etc. (the
orientation of the paper's Listing 1, Section 3.1), and every ring row of the
matrix is the identity (a Dirichlet ring held constant).  Works with float or
with Fraction entries (dtype=object) for exact arithmetic.
"""
from fractions import Fraction

import numpy as np


def shift(n, d, one):
    """n x n matrix with S[i, i+d] = one: (S v)[i] = v[i+d]."""
    m = np.zeros((n, n), dtype=object if isinstance(one, Fraction) else float)
    if m.dtype == object:
        m[:] = Fraction(0)
    for i in range(n):
        j = i + d
        if 0 <= j < n:
            m[i, j] = one
    return m


def full_matrix(nx, ny, w, exact=False):
    W, E, S, C, N = [Fraction(v) for v in w] if exact else [float(v) for v in w]
    one = Fraction(1) if exact else 1.0
    X, Y = nx + 2, ny + 2
    Ix = shift(X, 0, one)
    Iy = shift(Y, 0, one)
    A = (C * np.kron(Iy, Ix) + W * np.kron(Iy, shift(X, -1, one)) + E * np.kron(Iy, shift(X, +1, one))
         + S * np.kron(shift(Y, -1, one), Ix) + N * np.kron(shift(Y, +1, one), Ix))
    ring = np.ones((Y, X), dtype=bool)
    ring[1:-1, 1:-1] = False
    ring = ring.reshape(-1)
    Id = np.kron(Iy, Ix)
    A[ring, :] = Id[ring, :]
    return A


def apply_steps(A, u, steps):
    """u after `steps` applications of A (u has shape (ny+2, nx+2))."""
    v = u.reshape(-1)
    for _ in range(steps):
        v = A.dot(v)
    return v.reshape(u.shape)


def to_fraction(a):
    out = np.empty(a.shape, dtype=object)
    flat = a.reshape(-1)
    of = out.reshape(-1)
    for i, v in enumerate(flat):
        of[i] = Fraction(float(v))
    return out


def full_matrix_box(nx, ny, w, exact=False):
    """One step of the 3x3 box stencil (j2d9pt) as a matrix: the interior
    block is sum over dy, dx in {-1, 0, 1} of w[3*(dy+1) + (dx+1)] times
    (Dy^dy kron Dx^dx), where D^d reads the neighbour at offset d; ring rows
    are the identity."""
    ws = [Fraction(v) for v in w] if exact else [float(v) for v in w]
    one = Fraction(1) if exact else 1.0
    X, Y = nx + 2, ny + 2
    A = None
    for dy in (-1, 0, 1):
        for dx in (-1, 0, 1):
            term = ws[3 * (dy + 1) + (dx + 1)] * np.kron(shift(Y, dy, one), shift(X, dx, one))
            A = term if A is None else A + term
    ring = np.ones((Y, X), dtype=bool)
    ring[1:-1, 1:-1] = False
    ring = ring.reshape(-1)
    Id = np.kron(shift(Y, 0, one), shift(X, 0, one))
    A[ring, :] = Id[ring, :]
    return A
