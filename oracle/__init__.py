"""CPU oracle for the j2d5pt stencil -- test infrastructure only.

Plain, slow, obviously correct FP64 reference (C, no FMA, fixed left-to-right
summation order) that the CUDA library is checked against.  Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
it; the library itself never does.  It shares no code with the CUDA path.

Functions follow Zhang et al., GPGPU'23, Section 3.1 (Listing 1: the j2d5pt
update with weights W, E, S, C, N on x-1, x+1, y-1, centre, y+1; out-of-place
Jacobi), with a one-cell Dirichlet ring held constant (the paper is silent on
the boundary).  ``box_*`` are the same iteration for a second stencil shape,
the 3x3 box (j2d9pt): the paper treats j2d5pt as a case study of the method
(title, Section 1), whose step function does not depend on the shape.  The adjoint and weight gradient are the transpose and the
derivative of that map (linear algebra; the paper has no counterpart).

Parity pins: every function here is pinned by ``tests/test_oracle_pins.py``
(closed-form eigenmodes, exact rational arithmetic on dyadic inputs,
Kronecker-product matrix powers, invariants, dot-product and Euler
homogeneity identities).  No function is "parity unpinned".
"""
from .j2d5pt import (  # noqa: F401
    build, lib_path, step, run, run_f32, adjoint_step, adjoint_run, weight_grad,
    grad, dot, loss, max_threads, box_step, box_run, box_run_f32,
)
