"""Seeded random configurations of every kernel family.

Each case draws a grid size, a step count, a kernel family with its temporal
depth and tile shape, a dtype and a direction, and requires (1) bit-identical
results to the one-step kernel of the same plan (every family evaluates every
cell the same way) and (2) agreement with the oracle: within 1e-12 for FP64,
within the a-priori FP32 bound against the FP32 oracle.  Configurations a
family cannot run (a tile too small for the depth, a grid that does not fit
on chip) must be refused with J2D_ERR_UNSUPPORTED, never run wrongly.
"""
import numpy as np
import pytest

import oracle
from paper_2306_03336_gb300 import j2d5pt, synth
from tests.gpu_util import TOL_F64, f32_bound, rel_err

pytestmark = pytest.mark.gpu

N_CASES = 160


def _case(i):
    r = np.random.Generator(np.random.PCG64(2306033500 + i))
    nx = int(r.choice([1, 2, 3, 63, 64, 65, 127, 128, 129, 200, 257, 700]) if r.random() < 0.5 else r.integers(1, 701))
    ny = int(r.integers(1, 501))
    return dict(
        nx=nx, ny=ny,
        steps=int(r.choice([0, 1, 2, 3, 5, 8, 13, 21, 40])),
        algo=str(r.choice(["resident", "bands", "tiles"])),
        depth=int(r.choice([1, 2, 3, 4, 6, 8, 12, 16])),
        wx=int(r.choice([1, 2, 4, 8, 16])),
        dtype=str(r.choice(["f64", "f32"])),
        adjoint=bool(r.random() < 0.3),
        seed=2306033600 + i,
    )


@pytest.mark.parametrize("i", range(N_CASES))
def test_random_configuration(i):
    c = _case(i)
    nx, ny, steps, dt = c["nx"], c["ny"], c["steps"], c["dtype"]
    u0 = synth.field(nx, ny, c["seed"])
    w = synth.weights(c["seed"] + 1)
    p = j2d5pt.Plan(nx, ny, dt, w)
    src = p.to_device(u0 if dt == "f64" else u0.astype(np.float32))
    run = p.run_adjoint if c["adjoint"] else p.run
    # the one-step kernel of the same plan
    p.set("algo", "onestep")
    ref_dev = p.empty()
    run(src, ref_dev, steps)
    p.sync()
    ref = p.to_host(ref_dev)
    # the family under test
    p.set("algo", c["algo"]).set("depth", c["depth"]).set("tile_wx", c["wx"])
    out = p.empty()
    try:
        run(src, out, steps)
        p.sync()
    except j2d5pt.J2DError as e:
        assert e.status == j2d5pt.J2D_ERR_UNSUPPORTED, (c, str(e))
        p.close()
        pytest.skip("refused: %s" % e)
    got = p.to_host(out)
    p.close()
    assert np.array_equal(got, ref), (c, int(np.count_nonzero(got != ref)))
    if dt == "f64":
        ora = oracle.adjoint_run(u0, w, steps) if c["adjoint"] else oracle.run(u0, w, steps)
        assert rel_err(got, ora) <= TOL_F64, c
    elif not c["adjoint"]:
        ora = oracle.run_f32(u0.astype(np.float32).astype(np.float64), w, steps)
        assert rel_err(got, ora) <= f32_bound(steps), c


N_SKEWED = 60


@pytest.mark.parametrize("i", range(N_SKEWED))
def test_random_skewed_configuration(i):
    """The skewed serial tiles on seeded random sizes, depths and tile
    widths: bit-identical to the one-step kernel and within the oracle bars
    (forward runs; the schedule is forward only)."""
    r = np.random.Generator(np.random.PCG64(2306034100 + i))
    nx = int(r.choice([1, 2, 63, 64, 65, 127, 128, 129, 255, 256, 257, 700]) if r.random() < 0.5 else r.integers(1, 901))
    ny = int(r.integers(1, 601))
    steps = int(r.choice([1, 2, 3, 5, 8, 13, 21, 40]))
    depth = int(r.choice([1, 2, 3, 4, 6, 8, 12, 16, 24, 32]))
    wx = int(r.choice([1, 2, 4, 8, 16]))
    dt = str(r.choice(["f64", "f32"]))
    seed = 2306034200 + i
    u0 = synth.field(nx, ny, seed)
    w = synth.weights(seed + 1)
    p = j2d5pt.Plan(nx, ny, dt, w)
    src = p.to_device(u0 if dt == "f64" else u0.astype(np.float32))
    p.set("algo", "onestep")
    ref_dev = p.empty()
    p.run(src, ref_dev, steps)
    p.sync()
    ref = p.to_host(ref_dev)
    p.set("algo", "skewed").set("depth", depth).set("tile_wx", wx)
    out = p.empty()
    try:
        p.run(src, out, steps)
        p.sync()
    except j2d5pt.J2DError as e:
        assert e.status == j2d5pt.J2D_ERR_UNSUPPORTED, (nx, ny, steps, depth, wx, dt, str(e))
        p.close()
        pytest.skip("refused: %s" % e)
    got = p.to_host(out)
    p.close()
    assert np.array_equal(got, ref), (nx, ny, steps, depth, wx, dt, int(np.count_nonzero(got != ref)))
    if dt == "f64":
        assert rel_err(got, oracle.run(u0, w, steps)) <= TOL_F64
    else:
        assert rel_err(got, oracle.run_f32(u0.astype(np.float32).astype(np.float64), w, steps)) <= f32_bound(steps)


N_BATCHES = 12


@pytest.mark.parametrize("i", range(N_BATCHES))
def test_random_batch(i):
    """A batch of uneven grids with their own weights, one persistent launch:
    every grid bit-identical to its own single-grid one-step run."""
    r = np.random.Generator(np.random.PCG64(2306033800 + i))
    count = int(r.integers(1, 24))
    sizes = [(int(r.integers(1, 400)), int(r.integers(1, 300))) for _ in range(count)]
    dt = str(r.choice(["f64", "f32"]))
    steps = int(r.choice([1, 4, 9, 17]))
    depth = int(r.choice([1, 2, 4, 8]))
    wx = int(r.choice([1, 2, 4]))
    algo = "skewed" if i % 3 == 2 else "tiles"
    ws = np.stack([synth.weights(2306033900 + 10 * i + g) for g in range(count)])
    us = [synth.field(nx, ny, 2306034000 + 10 * i + g) for g, (nx, ny) in enumerate(sizes)]
    p = j2d5pt.Plan.batch(sizes, dt, ws).set("algo", algo).set("depth", depth).set("tile_wx", wx)
    srcs = [p.to_device(u.astype(p.np_dtype), g) for g, u in enumerate(us)]
    dsts = [p.empty(g) for g in range(count)]
    try:
        p.run_batched(srcs, dsts, steps)
        p.sync()
    except j2d5pt.J2DError as e:
        assert e.status == j2d5pt.J2D_ERR_UNSUPPORTED, str(e)
        p.close()
        pytest.skip("refused: %s" % e)
    outs = [p.to_host(d, g) for g, d in enumerate(dsts)]
    p.close()
    for g, (nx, ny) in enumerate(sizes):
        q = j2d5pt.Plan(nx, ny, dt, ws[g]).set("algo", "onestep")
        a, b = q.to_device(us[g].astype(q.np_dtype)), q.empty()
        q.run(a, b, steps)
        q.sync()
        assert np.array_equal(outs[g], q.to_host(b)), (i, g, nx, ny, dt, steps, depth, wx, algo)
        q.close()


N_STREAM = 60


@pytest.mark.parametrize("i", range(N_STREAM))
def test_random_stream_configuration(i):
    """The stream schedule on seeded random sizes (thin, ragged, a band or
    many), step counts around and across whole passes, and every depth it
    has a kernel for, forward, in place or not: bit-identical to the one-step
    kernel and within the oracle bounds."""
    r = np.random.Generator(np.random.PCG64(2306034200 + i))
    dt = str(r.choice(["f64", "f32"]))
    depth = int(r.choice([2, 3, 4, 6] if dt == "f64" else [4, 6, 8, 10, 12]))
    nx = int(r.choice([1, 2, 3, 59, 60, 61, 64, 112, 113, 128, 500]) if r.random() < 0.5 else r.integers(1, 901))
    ny = int(r.integers(1, 601))
    steps = int(r.choice([1, depth - 1, depth, depth + 1, 2 * depth, 3 * depth + 2, 17]))
    steps = max(steps, 1)
    alias = bool(r.random() < 0.25)
    seed = 2306034300 + i
    u0 = synth.field(nx, ny, seed)
    w = synth.weights(seed + 1)
    p = j2d5pt.Plan(nx, ny, dt, w)
    src = p.to_device(u0 if dt == "f64" else u0.astype(np.float32))
    p.set("algo", "onestep")
    ref_dev = p.empty()
    p.run(src, ref_dev, steps)
    p.sync()
    ref = p.to_host(ref_dev)
    p.set("algo", "stream").set("depth", depth)
    out = src if alias else p.empty()
    p.run(src, out, steps)
    p.sync()
    got = p.to_host(out)
    p.close()
    case = (dt, depth, nx, ny, steps, alias)
    assert np.array_equal(got, ref), (case, int(np.count_nonzero(got != ref)))
    if dt == "f64":
        assert rel_err(got, oracle.run(u0, w, steps)) <= TOL_F64, case
    else:
        assert rel_err(got, oracle.run_f32(u0.astype(np.float32).astype(np.float64), w, steps)) <= f32_bound(steps), case
