"""Parity at the full workload sizes, in the launch configurations the
benchmark times.

- FP64 2048 x 1536, 1000 steps: every kernel family against the oracle on the
  whole grid (the oracle runs it in well under a second on the host cores).
- FP64 and FP32 16384 x 16384, 1000 steps: sampled cells against the oracle.
  A cell's value after T steps depends only on the initial cells within
  distance T of it, so the oracle evaluates it exactly on the window of radius
  T+1 around the cell (window edge held constant: its changes cannot reach the
  centre within T steps).
"""
import numpy as np
import pytest

import oracle
from paper_2306_03336_gb300 import j2d5pt, synth
from tests.gpu_util import TOL_F64, cell_rel_err, f32_bound, rel_err

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


@pytest.mark.parametrize("algo,depth", [("resident", 0), ("bands", 32), ("bands", 8), ("tiles", 4), ("onestep", 0)])
def test_headline_workload_full_grid(headline, algo, depth):
    u0, w, steps, ref = headline
    p, dst = _run(u0, w, steps, "f64", algo, depth)
    got = p.to_host(dst)
    p.close()
    assert rel_err(got, ref) <= TOL_F64
    assert cell_rel_err(got, ref) <= TOL_F64


def _window_value(u0, w, steps, y, x):
    H, W = u0.shape
    r = steps + 1
    y0, y1 = max(0, y - r), min(H - 1, y + r)
    x0, x1 = max(0, x - r), min(W - 1, x + r)
    win = np.ascontiguousarray(u0[y0:y1 + 1, x0:x1 + 1])
    out = oracle.run(win, w, steps, threads=oracle.max_threads())
    return out[y - y0, x - x0]


def test_16384_workloads_sampled_cells():
    import torch
    n, steps = 16384, 1000
    u0 = synth.field(n, n, synth.data_seed(1))
    w = synth.weights(synth.weight_seed(1))
    # interior cells far from the ring, one near a corner, and ring-adjacent ones
    cells = [(1, 1), (n, n), (3000, 9000), (1, 5000), (12000, 2)]
    refs = [_window_value(u0, w, steps, y, x) for (y, x) in cells]
    for algo, depth, wx in (("onestep", 0, 0), ("tiles", 4, 2), ("bands", 8, 0)):
        p, dst = _run(u0, w, steps, "f64", algo, depth, wx)
        v = p.view(dst)
        for (y, x), ref in zip(cells, refs):
            assert abs(float(v[y, x]) - ref) <= TOL_F64 * abs(ref), (algo, y, x)
        p.close()
        del dst
        torch.cuda.empty_cache()
    p, dst = _run(u0, w, steps, "f32", "tiles", 16, 2)
    v = p.view(dst)
    for (y, x), ref in zip(cells, refs):
        assert abs(float(v[y, x]) - ref) <= f32_bound(steps) * abs(ref), ("f32", y, x)
    p.close()
