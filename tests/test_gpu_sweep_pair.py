"""Two time steps per sweep (FP32 tiles, forward).

With J2D_OPT_SWEEP_STEPS = 2 a strip reads its neighbours' cells two deep,
evaluates the first step on the ring around itself as the owning strips do,
and sweeps its rows once for both steps.  Every cell must come out bit-identical
to the one-step kernel and to the single-step tiles, across tile shapes, odd
and even depths (an odd depth ends with one single step), ragged grids whose
last strip has one row, strips with dead columns, one-column grids, batches,
and the oracle's FP32 bound.
"""
import numpy as np
import pytest

import oracle
from paper_2306_03336_gb300 import j2d5pt, synth
from tests.gpu_util import f32_bound, rel_err

pytestmark = pytest.mark.gpu


def _pair_rows():
    p = j2d5pt.Plan(4096, 4096, "f32", synth.weights(1)).set("algo", "tiles").set("sweep_steps", 2)
    d = dict(kv.split("=") for kv in p.describe().split())
    p.close()
    assert d["sweep"] == "2"
    return int(d["rows"])


def _run(p, src, steps, **opts):
    for k, v in opts.items():
        p.set(k, v)
    out = p.empty()
    p.run(src, out, steps)
    p.sync()
    return p.to_host(out)


SIZES = [(1, 1), (1, 40), (5, 3), (128, 27), (129, 28), (130, 55), (257, 109), (300, 200), (513, 82), (700, 300)]


@pytest.mark.parametrize("nx,ny", SIZES)
@pytest.mark.parametrize("wx", [1, 2, 4, 16])
def test_pair_bit_identical(nx, ny, wx):
    u0 = synth.field(nx, ny, 2306035000 + nx * 7 + ny)
    w = synth.weights(2306035001 + wx)
    p = j2d5pt.Plan(nx, ny, "f32", w)
    src = p.to_device(u0.astype(np.float32))
    for steps, depth in ((7, 2), (9, 4), (10, 3), (5, 5), (33, 16), (1, 1)):
        ref = _run(p, src, steps, algo="onestep")
        for sweep in (1, 2):
            try:
                got = _run(p, src, steps, algo="tiles", depth=depth, tile_wx=wx, sweep_steps=sweep)
            except j2d5pt.J2DError as e:
                # a tile too small for the depth is refused, never run wrongly
                assert e.status == j2d5pt.J2D_ERR_UNSUPPORTED, str(e)
                continue
            bad = np.argwhere(got != ref)
            assert bad.size == 0, "nx=%d ny=%d wx=%d steps=%d depth=%d sweep=%d: %d cells differ, first (y, x) = %s" % (
                nx, ny, wx, steps, depth, sweep, len(bad), tuple(bad[0]))
    p.close()


def test_pair_last_strip_one_row():
    """ny = rows + 1: the second strip of the tile has a single row, and the
    strip above it reads that row and the ring row below it."""
    r = _pair_rows()
    nx, ny = 300, r + 1
    u0 = synth.field(nx, ny, 2306035100)
    w = synth.weights(2306035101)
    p = j2d5pt.Plan(nx, ny, "f32", w)
    src = p.to_device(u0.astype(np.float32))
    ref = _run(p, src, 12, algo="onestep")
    for wx in (1, 2, 4):
        got = _run(p, src, 12, algo="tiles", depth=6, tile_wx=wx, sweep_steps=2)
        assert np.array_equal(got, ref), wx
    p.close()


def test_pair_against_oracle():
    nx, ny, steps = 600, 450, 40
    u0 = synth.field(nx, ny, 2306035200)
    w = synth.weights(2306035201)
    p = j2d5pt.Plan(nx, ny, "f32", w).set("algo", "tiles").set("depth", 8).set("tile_wx", 2)
    assert p.get("sweep_steps") == 2
    src = p.to_device(u0.astype(np.float32))
    got = _run(p, src, steps)
    p.close()
    ora = oracle.run_f32(u0.astype(np.float32).astype(np.float64), w, steps)
    assert rel_err(got, ora) <= f32_bound(steps)


def test_pair_batch():
    """A batch of uneven FP32 grids: each grid bit-identical to its own
    single-grid one-step run."""
    r = np.random.Generator(np.random.PCG64(2306035300))
    sizes = [(int(r.integers(1, 500)), int(r.integers(1, 300))) for _ in range(9)]
    ws = np.stack([synth.weights(2306035310 + g) for g in range(len(sizes))])
    us = [synth.field(nx, ny, 2306035320 + g).astype(np.float32) for g, (nx, ny) in enumerate(sizes)]
    p = j2d5pt.Plan.batch(sizes, "f32", ws).set("algo", "tiles").set("depth", 4).set("tile_wx", 2)
    assert p.get("sweep_steps") == 2
    srcs = [p.to_device(u, g) for g, u in enumerate(us)]
    dsts = [p.empty(g) for g in range(len(sizes))]
    p.run_batched(srcs, dsts, 11)
    p.sync()
    outs = [p.to_host(d, g) for g, d in enumerate(dsts)]
    p.close()
    for g, (nx, ny) in enumerate(sizes):
        q = j2d5pt.Plan(nx, ny, "f32", ws[g]).set("algo", "onestep")
        a, b = q.to_device(us[g]), q.empty()
        q.run(a, b, 11)
        q.sync()
        assert np.array_equal(outs[g], q.to_host(b)), (g, nx, ny)
        q.close()


def test_sweep_steps_option():
    p = j2d5pt.Plan(64, 64, "f32", synth.weights(3))
    assert p.get("sweep_steps") == 2
    p.set("sweep_steps", 1)
    assert p.get("sweep_steps") == 1
    with pytest.raises(j2d5pt.J2DError):
        p.set("sweep_steps", 3)
    p.close()
