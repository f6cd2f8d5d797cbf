"""The allocation-free weight-gradient entry point (j2d5pt_weight_grad_noalloc).

It serves callers that cannot call cudaMalloc -- code inside a CUDA-graph
stream capture, code whose device memory belongs to a framework's caching
allocator, latency-bound loops that cannot take cudaFree's device-wide
synchronisation -- by keeping its scratch in a fixed device array inside the
library.  This test calls it through the C ABI twice in a row, a large grid and then
a smaller one (the array keeps the previous call's contents), and checks each
result against the plan-based entry point j2d5pt_weight_grad on the same
grid; it also checks that an oversize grid is refused.
The file name makes pytest collect it last.
"""
import numpy as np
import pytest

from paper_2306_03336_gb300 import j2d5pt, synth
from tests.gpu_util import TOL_F64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _plan_reference(nx, ny, dtype, w, seed):
    """Fields of one grid and its weight gradient from the plan-based entry point."""
    import torch
    p = j2d5pt.Plan(nx, ny, dtype, w)
    u = p.to_device(synth.field(nx, ny, seed))
    lam = p.to_device(synth.field(nx, ny, seed + 1))
    ref = torch.zeros(5, dtype=torch.float64, device="cuda")
    p.weight_grad(u, lam, ref)
    p.sync()
    p.close()
    return u, lam, ref


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_noalloc_matches_plan_entry_on_two_calls(dtype):
    """A large grid, then a smaller one with other fields: the second call
    uses fewer partial-sum blocks than the first left in the shared array, so
    a reduction that read past its own blocks would pick up stale sums."""
    import torch
    code = j2d5pt.J2D_F64 if dtype == "f64" else j2d5pt.J2D_F32
    w = synth.weights(7)
    for nx, ny, seed in ((1517, 1263, 11), (517, 263, 21)):
        u, lam, ref = _plan_reference(nx, ny, dtype, w, seed)
        dw = torch.zeros(5, dtype=torch.float64, device="cuda")
        j2d5pt.j2d5pt_weight_grad_noalloc(nx, ny, code, u, lam, dw)
        torch.cuda.synchronize()
        assert (dw - ref).abs().max().item() <= TOL_F64 * ref.abs().max().item(), (nx, ny)


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch
    u = torch.zeros(16, dtype=torch.float64, device="cuda")
    dw = torch.zeros(5, dtype=torch.float64, device="cuda")
    with pytest.raises(j2d5pt.J2DError) as e:
        j2d5pt.j2d5pt_weight_grad_noalloc(200000, 200000, j2d5pt.J2D_F64, u, u, dw)
    assert e.value.status == j2d5pt.J2D_ERR_ARG
    assert "partial-sum blocks" in str(e.value)
