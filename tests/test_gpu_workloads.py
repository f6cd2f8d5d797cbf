"""Parity at the full workload sizes, in the launch configurations the
benchmark times.

- FP64 2048 x 1536, 1000 steps: every kernel family against the oracle on the
  whole grid (the oracle runs it in well under a second on the host cores).
- FP64 and FP32 16384 x 16384, 1000 steps, and the paper's evaluation domain
  8592 x 8328 (Section 4, Figure 2): the plan the benchmark uses (autotuned)
  and fixed kernel choices, every cell of every grid bit for bit against the
  one-step kernel on the device (the blocked kernels evaluate each cell with
  the same operands in the same order, so tiling cannot change a bit), and
  blocks of 300 x 300 cells -- the corners with their ring-adjacent cells,
  the middle, the middle of two edges, each holding tile seams and CTA-group
  edges in both axes -- against the oracle.  A cell's value after T steps
  depends only on the initial cells within distance T of it, so the oracle
  evaluates a block exactly on the block plus a margin of T+1 cells.
"""
import numpy as np
import pytest

import oracle
from paper_2306_03336_gb300 import j2d5pt, synth
from tests.gpu_util import TOL_F64, blocks_for, cell_rel_err, f32_bound, rel_err, window_block

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _run(u0, w, steps, dtype, algo, depth=0, wx=0):
    ny, nx = u0.shape[0] - 2, u0.shape[1] - 2
    p = j2d5pt.Plan(nx, ny, dtype, w).set("algo", algo)
    if depth:
        p.set("depth", depth)
    if wx:
        p.set("tile_wx", wx)
    src = p.to_device(u0 if dtype == "f64" else u0.astype(np.float32))
    dst = p.empty()
    p.run(src, dst, steps)
    p.sync()
    return p, dst


@pytest.fixture(scope="module")
def headline():
    nx, ny, steps = 2048, 1536, 1000
    u0 = synth.field(nx, ny, synth.data_seed(1))
    w = synth.weights(synth.weight_seed(1))
    return u0, w, steps, oracle.run(u0, w, steps, threads=oracle.max_threads())


@pytest.mark.parametrize("algo,depth", [("resident", 0), ("bands", 32), ("bands", 8), ("tiles", 4), ("onestep", 0),
                                        ("stream", 2), ("stream", 6)])
def test_headline_workload_full_grid(headline, algo, depth):
    u0, w, steps, ref = headline
    p, dst = _run(u0, w, steps, "f64", algo, depth)
    got = p.to_host(dst)
    p.close()
    assert rel_err(got, ref) <= TOL_F64
    assert cell_rel_err(got, ref) <= TOL_F64


def _full_size_case(u0, w, steps, dtype, variants, tol):
    """Run the one-step kernel, the autotuned plan and each (algo, depth, wx)
    variant on u0; every result must equal the one-step result bit for bit,
    and the oracle blocks must agree within `tol` (relative to each cell)."""
    import torch
    ny, nx = u0.shape[0] - 2, u0.shape[1] - 2
    ref_plan = j2d5pt.Plan(nx, ny, dtype, w).set("algo", "onestep")
    src = ref_plan.to_device(u0 if dtype == "f64" else u0.astype(np.float32))
    ref = ref_plan.empty()
    ref_plan.run(src, ref, steps)
    ref_plan.sync()
    ref_plan.close()
    blocks = blocks_for(ny, nx)
    expect = [window_block(oracle, u0 if dtype == "f64" else u0.astype(np.float32).astype(np.float64), w,
                           steps, *b) for b in blocks]
    tried = []
    for variant in [("autotuned", 0, 0)] + list(variants):
        algo, depth, wx = variant
        p = j2d5pt.Plan(nx, ny, dtype, w)
        dst = p.empty()
        if algo == "autotuned":
            p.autotune(src, dst, steps)
        else:
            p.set("algo", algo)
            if depth:
                p.set("depth", depth)
            if wx:
                p.set("tile_wx", wx)
        dst.zero_()
        p.run(src, dst, steps)
        p.sync()
        tried.append(p.describe())
        assert torch.equal(p.view(dst), p.view(ref)), ("not bit-identical to the one-step kernel", p.describe())
        v = p.view(dst)
        for (y0, y1, x0, x1), e in zip(blocks, expect):
            got = v[y0:y1, x0:x1].double().cpu().numpy()
            err = np.abs(got - e) / np.maximum(np.abs(e), 1e-300)
            assert err.max() <= tol, (p.describe(), (y0, x0), float(err.max()))
        p.close()
        del dst
        torch.cuda.empty_cache()
    return tried


def test_16384_f64_full_grid_bitwise_and_oracle_blocks():
    n, steps = 16384, 1000
    u0 = synth.field(n, n, synth.data_seed(1))
    w = synth.weights(synth.weight_seed(1))
    _full_size_case(u0, w, steps, "f64", [("tiles", 4, 4), ("tiles", 4, 2), ("bands", 8, 0), ("skewed", 8, 4),
                                          ("skewed", 16, 8), ("stream", 2, 0), ("stream", 3, 0)], TOL_F64)


def test_16384_f32_full_grid_bitwise_and_oracle_blocks():
    n, steps = 16384, 1000
    u0 = synth.field(n, n, synth.data_seed(1))
    w = synth.weights(synth.weight_seed(1))
    _full_size_case(u0, w, steps, "f32", [("tiles", 16, 2), ("tiles", 16, 4), ("skewed", 16, 4), ("skewed", 24, 8),
                                          ("stream", 8, 0), ("stream", 12, 0)], f32_bound(steps))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_paper_domain_8592x8328(dtype):
    """The paper's evaluation domain (Section 4, Figure 2: 8592 x 8328 run,
    8192^2 counted as the valid domain), with the benchmark's seed."""
    nx, ny, steps = 8592, 8328, 1000
    u0 = synth.field(nx, ny, synth.data_seed(1) + 20)
    w = synth.weights(synth.weight_seed(1))
    tol = TOL_F64 if dtype == "f64" else f32_bound(steps)
    _full_size_case(u0, w, steps, dtype, [("tiles", 4, 4), ("skewed", 8, 4), ("stream", 2, 0)] if dtype == "f64"
                    else [("tiles", 16, 4), ("skewed", 16, 4), ("stream", 8, 0)], tol)
