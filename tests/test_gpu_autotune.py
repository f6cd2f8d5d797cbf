"""The autotuner (j2d5pt_autotune / j2d5pt_autotune_batched) and its cache
file (J2D_TUNE_CACHE).

- A tuned plan still computes the same map: the oracle within the FP64 bar,
  bit for bit against the one-step kernel.
- The cache round-trips: the first tuning appends one whitespace-free key
  and the choice; a second plan of the same key reads it back without
  appending; a choice written into the file by hand is the one a plan adopts.
- The batched tuner picks a configuration that keeps every grid bit-identical
  to its single-grid one-step run.
"""
import numpy as np
import pytest

import oracle
from paper_2306_03336_gb300 import j2d5pt, synth
from tests.gpu_util import TOL_F64, f32_bound, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


@pytest.fixture
def no_cache(monkeypatch):
    monkeypatch.delenv("J2D_TUNE_CACHE", raising=False)


def _onestep(nx, ny, dtype, w, src, steps):
    q = j2d5pt.Plan(nx, ny, dtype, w).set("algo", "onestep")
    out = q.empty()
    q.run(src, out, steps)
    q.sync()
    q.close()
    return out


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_tuned_plan_matches_oracle_and_onestep(no_cache, dtype):
    import torch
    nx, ny, steps = 1000, 700, 64
    u0 = synth.field(nx, ny, 701)
    w = synth.weights(702)
    p = j2d5pt.Plan(nx, ny, dtype, w)
    src = p.to_device(u0 if dtype == "f64" else u0.astype(np.float32))
    dst = p.empty()
    desc = p.autotune(src, dst, steps)
    assert "algo=" in desc
    dst.zero_()
    p.run(src, dst, steps)
    p.sync()
    got = p.to_host(dst)
    if dtype == "f64":
        assert rel_err(got, oracle.run(u0, w, steps, threads=oracle.max_threads())) <= TOL_F64
    else:
        ref = oracle.run(u0.astype(np.float32).astype(np.float64), w, steps, threads=oracle.max_threads())
        assert rel_err(got, ref) <= f32_bound(steps)
    assert torch.equal(p.view(dst), p.view(_onestep(nx, ny, dtype, w, src, steps)))
    p.close()


def _choice(p):
    return p.get("algo"), p.get("depth"), p.get("tile_wx")


def test_tune_cache_round_trip(tmp_path, monkeypatch):
    cache = tmp_path / "tune.txt"
    monkeypatch.setenv("J2D_TUNE_CACHE", str(cache))
    nx, ny, steps = 900, 600, 48
    u0 = synth.field(nx, ny, 711)
    w = synth.weights(712)
    a = j2d5pt.Plan(nx, ny, "f64", w)
    src, dst = a.to_device(u0), a.empty()
    a.autotune(src, dst, steps)
    lines = cache.read_text().splitlines()
    assert len(lines) == 1
    fields = lines[0].split()
    assert len(fields) == 4, lines[0]  # key without whitespace, algo, depth, tile_wx
    key = fields[0]
    assert tuple(int(f) for f in fields[1:]) == _choice(a)
    # a second plan with the same key reads the cached choice and appends nothing
    b = j2d5pt.Plan(nx, ny, "f64", w)
    b.autotune(src, dst, steps)
    assert _choice(b) == _choice(a)
    assert len(cache.read_text().splitlines()) == 1
    # a choice written by hand under the same key is the one adopted
    forced = (j2d5pt.ALGO["tiles"], 6, 2) if _choice(a) != (j2d5pt.ALGO["tiles"], 6, 2) else (j2d5pt.ALGO["bands"], 5, 0)
    cache.write_text("%s %d %d %d\n" % ((key,) + forced))
    c = j2d5pt.Plan(nx, ny, "f64", w)
    c.autotune(src, dst, steps)
    assert _choice(c) == forced
    assert ("algo=tiles" if forced[0] == j2d5pt.ALGO["tiles"] else "algo=bands") in c.describe()
    dst.zero_()
    c.run(src, dst, steps)
    c.sync()
    assert rel_err(c.to_host(dst), oracle.run(u0, w, steps, threads=oracle.max_threads())) <= TOL_F64
    # a different step-count bucket is another key: tuned afresh and appended
    d = j2d5pt.Plan(nx, ny, "f64", w)
    d.autotune(src, dst, 300)
    assert len(cache.read_text().splitlines()) == 2
    for p in (a, b, c, d):
        p.close()


def test_autotune_batched(no_cache):
    import torch
    sizes = [(300, 200), (64, 64), (130, 7), (1024, 64), (257, 331), (95, 95)]
    steps = 40
    w = np.stack([synth.weights(720 + i) for i in range(len(sizes))])
    us = [synth.field(nx, ny, 730 + i) for i, (nx, ny) in enumerate(sizes)]
    p = j2d5pt.Plan.batch(sizes, "f64", w)
    srcs = [p.to_device(u, i) for i, u in enumerate(us)]
    dsts = [p.empty(i) for i in range(len(sizes))]
    desc = p.autotune_batched(srcs, dsts, steps)
    assert any("algo=%s " % a in desc + " " for a in ("tiles", "skewed", "resident")), desc
    for d in dsts:
        d.zero_()
    p.run_batched(srcs, dsts, steps)
    p.sync()
    for i, (nx, ny) in enumerate(sizes):
        assert torch.equal(p.view(dsts[i], i), p.view(_onestep(nx, ny, "f64", w[i], srcs[i], steps), i))
        assert rel_err(p.to_host(dsts[i], i), oracle.run(us[i], w[i], steps)) <= TOL_F64
    p.close()


def test_autotune_argument_errors():
    p = j2d5pt.Plan(64, 64, "f64", synth.weights(1))
    a = p.empty()
    with pytest.raises(j2d5pt.J2DError) as e:
        p.autotune(a, a, 0)
    assert e.value.status == j2d5pt.J2D_ERR_ARG
    p.close()
