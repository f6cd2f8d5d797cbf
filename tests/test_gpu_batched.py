"""Batched grids of uneven sizes with their own weights, advanced together in
one persistent launch, plain and captured in a CUDA graph; every grid against
the oracle and bit for bit against the one-step kernel.  The tiled, skewed
and grouped-resident schedules (the grids in waves, each wave on chip for
all steps), the last also with few CTAs so that a batch takes many waves."""
import numpy as np
import pytest

import oracle
from paper_2306_03336_gb300 import j2d5pt, synth
from tests.gpu_util import TOL_F64, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


SIZES = [(1, 1), (300, 200), (64, 64), (130, 7), (7, 130), (257, 331), (1024, 64), (64, 1024), (95, 95), (513, 2)]


def _batch(sizes, dtype, steps, depth, wx, graph=False, replays=1, algo="tiles", ctas=0, expect=None):
    w = np.stack([synth.weights(400 + i) for i in range(len(sizes))])
    us = [synth.field(nx, ny, 500 + i) for i, (nx, ny) in enumerate(sizes)]
    p = j2d5pt.Plan.batch(sizes, dtype, w).set("algo", algo).set("depth", depth).set("tile_wx", wx)
    if ctas:
        p.set("ctas", ctas)
    if graph:
        p.set("graph", 1)
    if expect:
        assert "algo=%s " % expect in p.describe() + " ", p.describe()
    srcs = [p.to_device(u.astype(p.np_dtype), i) for i, u in enumerate(us)]
    dsts = [p.empty(i) for i in range(len(sizes))]
    for _ in range(replays):
        for d in dsts:
            d.zero_()
        p.run_batched(srcs, dsts, steps)
        p.sync()
    outs = [p.to_host(d, i) for i, d in enumerate(dsts)]
    p.close()
    return us, w, outs


@pytest.mark.parametrize("algo,depth,wx", [("tiles", 4, 2), ("tiles", 7, 1), ("tiles", 3, 4), ("skewed", 4, 2),
                                           ("skewed", 6, 4), ("skewed", 13, 8), ("resident", 0, 0)])
def test_batched_against_oracle(algo, depth, wx):
    steps = 13
    us, w, outs = _batch(SIZES, "f64", steps, depth, wx, algo=algo, expect=algo)
    for u, wi, got in zip(us, w, outs):
        assert rel_err(got, oracle.run(u, wi, steps)) <= TOL_F64


def _onestep_single(sizes, us, w, dtype, steps):
    outs = []
    for (nx, ny), u, wi in zip(sizes, us, w):
        p = j2d5pt.Plan(nx, ny, dtype, wi).set("algo", "onestep")
        src = p.to_device(u.astype(p.np_dtype))
        dst = p.empty()
        p.run(src, dst, steps)
        outs.append(p.to_host(dst))
        p.close()
    return outs


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("algo,ctas", [("tiles", 0), ("resident", 0), ("resident", 1), ("resident", 3), ("resident", 37)])
def test_batched_bitwise_equal_to_single_grid_onestep(dtype, algo, ctas):
    # with 1 or 3 CTAs (16 or 48 strips) the grouped-resident batch runs in
    # many waves, the large grids with tall strips in waves of their own (the
    # grids kept are those that fit 16 * ctas strips of 21 rows by themselves)
    steps = 9
    sizes = [s for s in SIZES if not ctas or (s[0] + 63) // 64 * ((s[1] + 20) // 21) <= 16 * ctas]
    us, w, outs = _batch(sizes, dtype, steps, 4, 2, algo=algo, ctas=ctas, expect=algo)
    for i, (a, b) in enumerate(zip(_onestep_single(sizes, us, w, dtype, steps), outs)):
        assert np.array_equal(a, b), (i, sizes[i])


def test_grouped_resident_many_small_grids():
    # 60 small grids share CTAs (several grids in one CTA's 16 strips)
    sizes = [(1 + (7 * i) % 150, 1 + (11 * i) % 90) for i in range(60)]
    steps = 17
    us, w, outs = _batch(sizes, "f64", steps, 0, 0, algo="resident", ctas=5, expect="resident")
    for i, (a, b) in enumerate(zip(_onestep_single(sizes, us, w, "f64", steps), outs)):
        assert np.array_equal(a, b), (i, sizes[i])
    for i in (0, 13, 59):
        assert rel_err(outs[i], oracle.run(us[i], w[i], steps)) <= TOL_F64


def test_grouped_resident_falls_back_when_a_grid_does_not_fit():
    # a grid too large for the GPU's strips by itself: RESIDENT resolves to tiles
    p = j2d5pt.Plan.batch([(64, 64), (4096, 4096)], "f64", np.stack([synth.weights(1), synth.weights(2)]))
    p.set("algo", "resident").set("ctas", 8)
    assert "algo=tiles" in p.describe()
    p.close()


@pytest.mark.parametrize("algo", ["tiles", "skewed", "resident"])
def test_batched_cuda_graph_replay(algo):
    steps = 10
    _, _, plain = _batch(SIZES, "f64", steps, 4, 2, algo=algo)
    _, _, graph = _batch(SIZES, "f64", steps, 4, 2, graph=True, replays=3, algo=algo)
    for a, b in zip(plain, graph):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("algo", ["autotuned", "resident", "tiles"])
def test_batched_workload_256_grids_all(algo):
    """The benchmark batch (256 grids, sides uniform in [64, 1024], 200 steps)
    in the benchmark's launch configuration (autotuned, CUDA graph) and in the
    grouped-resident and tiled schedules: every grid bit for bit against its
    own single-grid one-step run on the device, and a sample of grids against
    the oracle."""
    import torch
    cfg = synth.WORKLOADS["j2d5pt_f64_batch256_200"]
    sizes = synth.batch_sizes(cfg["count"], synth.data_seed(cfg["index"]), cfg["lo"], cfg["hi"])
    w = np.stack([synth.weights(synth.weight_seed(cfg["index"]) + i) for i in range(len(sizes))])
    p = j2d5pt.Plan.batch(sizes, "f64", w)
    us = [synth.field(nx, ny, synth.data_seed(cfg["index"]) + 10 + i) for i, (nx, ny) in enumerate(sizes)]
    srcs = [p.to_device(u, i) for i, u in enumerate(us)]
    dsts = [p.empty(i) for i in range(len(sizes))]
    if algo == "autotuned":
        p.autotune_batched(srcs, dsts, cfg["steps"])
    else:
        p.set("algo", algo)
    p.set("graph", 1)
    for _ in range(2):  # capture, then replay
        for d in dsts:
            d.zero_()
        p.run_batched(srcs, dsts, cfg["steps"])
        p.sync()
    for i, (nx, ny) in enumerate(sizes):
        q = j2d5pt.Plan(nx, ny, "f64", w[i]).set("algo", "onestep")
        out = q.empty()
        q.run(srcs[i], out, cfg["steps"])
        q.sync()
        assert torch.equal(q.view(out), p.view(dsts[i], i)), (i, nx, ny, p.describe())
        q.close()
    for i in (0, 17, 100, 255):
        ref = oracle.run(us[i], w[i], cfg["steps"], threads=oracle.max_threads())
        assert rel_err(p.to_host(dsts[i], i), ref) <= TOL_F64
    p.close()


def test_single_grid_graph_option():
    nx, ny, steps = 200, 150, 12
    u0 = synth.field(nx, ny, 601)
    w = synth.weights(602)
    p = j2d5pt.Plan(nx, ny, "f64", w).set("graph", 1)
    src = p.to_device(u0)
    dst = p.empty()
    for _ in range(3):
        dst.zero_()
        p.run(src, dst, steps)
        p.sync()
        assert rel_err(p.to_host(dst), oracle.run(u0, w, steps)) <= TOL_F64
    # new weights drop the graph
    w2 = synth.weights(603)
    p.set_weights(w2)
    p.run(src, dst, steps)
    p.sync()
    assert rel_err(p.to_host(dst), oracle.run(u0, w2, steps)) <= TOL_F64
    p.close()


@pytest.mark.parametrize("algo", ["onestep", "resident", "tiles", "skewed"])
def test_graph_with_timing(algo):
    """Timing events are not recorded inside the graph capture, so a plan
    with both options runs, replays and reports a kernel time afterwards."""
    nx, ny, steps = 200, 150, 12
    u0 = synth.field(nx, ny, 611)
    w = synth.weights(612)
    p = j2d5pt.Plan(nx, ny, "f64", w).set("algo", algo).set("graph", 1).set("timing", 1)
    src = p.to_device(u0)
    dst = p.empty()
    for _ in range(3):
        p.run(src, dst, steps)
        p.sync()
        assert p.kernel_time() > 0
    assert rel_err(p.to_host(dst), oracle.run(u0, w, steps)) <= TOL_F64
    p.close()
