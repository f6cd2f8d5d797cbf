"""GB300-native deep temporal blocking for the 2D Jacobi 5-point stencil (j2d5pt).

The compute path is the CUDA library ``libj2d5pt.so`` (hand-written sm_103a
kernels behind a C ABI, declared in ``include/j2d5pt.h``); this package holds
its thin ctypes binding, the torch autograd wrapper and the seeded input
generators.
"""
