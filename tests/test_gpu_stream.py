"""The STREAM schedule (temporal blocking in the register file): bit for bit
against the one-step kernel for every steps-per-pass kernel, on ragged, thin
and tall grids (many runs per band, so the runs' overlapped seams in y are
crossed, and several bands, so the seams in x are), step counts below, at and
above a pass (the first pass taking the remainder), in place and out of place;
against the oracle (dyadic inputs bit-identical); and its argument errors."""
import numpy as np
import pytest

import oracle
from paper_2306_03336_gb300 import j2d5pt, synth
from tests.gpu_util import TOL_F64, f32_bound, rel_err

pytestmark = pytest.mark.gpu

DEPTHS = {"f64": [2, 3, 4, 6], "f32": [4, 6, 8, 10, 12]}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def run(u0, w, steps, dtype, algo, depth=None, alias=False):
    ny, nx = u0.shape[0] - 2, u0.shape[1] - 2
    p = j2d5pt.Plan(nx, ny, dtype, w).set("algo", algo)
    if depth:
        p.set("depth", depth)
    src = p.to_device(u0)
    dst = src if alias else p.empty()
    p.run(src, dst, steps)
    p.sync()
    out = p.to_host(dst)
    p.close()
    return out


def field(nx, ny, seed, dtype):
    u0 = synth.field(nx, ny, seed)
    return u0.astype(np.float32) if dtype == "f32" else u0


SIZES = [(1, 1), (5, 3), (3, 700), (700, 3), (129, 257), (1000, 333), (200, 3000)]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("nx,ny", SIZES)
def test_bitwise_equal_to_onestep(dtype, nx, ny):
    w = synth.weights(500 + nx)
    u0 = field(nx, ny, 501 + ny, dtype)
    for depth in DEPTHS[dtype]:
        for steps in sorted({1, depth - 1, depth, 2 * depth + 1, 13}):
            if steps < 1:
                continue
            ref = run(u0, w, steps, dtype, "onestep")
            got = run(u0, w, steps, dtype, "stream", depth)
            assert np.array_equal(got, ref), (dtype, nx, ny, depth, steps)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_in_place(dtype):
    nx, ny = 333, 190
    w = synth.weights(510)
    u0 = field(nx, ny, 511, dtype)
    depth = DEPTHS[dtype][1]
    for steps in (1, depth, depth + 1, 2 * depth, 3 * depth - 1):  # odd and even pass counts
        ref = run(u0, w, steps, dtype, "onestep")
        assert np.array_equal(run(u0, w, steps, dtype, "stream", depth, alias=True), ref), (dtype, steps)


def test_against_oracle_f64():
    nx, ny, steps = 611, 402, 50
    w = synth.weights(520)
    u0 = synth.field(nx, ny, 521)
    ref = oracle.run(u0, w, steps, threads=4)
    for depth in DEPTHS["f64"]:
        assert rel_err(run(u0, w, steps, "f64", "stream", depth), ref) <= TOL_F64, depth


def test_against_oracle_f32():
    nx, ny, steps = 611, 402, 50
    w = synth.weights(522)
    u0 = synth.field(nx, ny, 523)
    ref = oracle.run(u0.astype(np.float32).astype(np.float64), w, steps, threads=4)
    for depth in DEPTHS["f32"]:
        assert rel_err(run(u0.astype(np.float32), w, steps, "f32", "stream", depth), ref) <= f32_bound(steps)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_dyadic_bit_identical_to_oracle(dtype):
    # dyadic data and weights stay exact for 6 steps in binary64, 4 in binary32
    nx, ny, steps = 300, 140, 6 if dtype == "f64" else 4
    w = synth.dyadic_weights()
    u0 = synth.dyadic_field(nx, ny, 530)
    ref = oracle.run(u0, w, steps)
    for depth in DEPTHS[dtype]:
        got = run(u0.astype(np.float32) if dtype == "f32" else u0, w, steps, dtype, "stream", depth)
        assert np.array_equal(got, ref), depth


@pytest.mark.parametrize("int_path", [0, 1])
def test_int_path_option(int_path):
    nx, ny, steps = 257, 300, 9
    w = synth.weights(540)
    u0 = synth.field(nx, ny, 541)
    refs = []
    for algo in ("onestep", "stream"):
        p = j2d5pt.Plan(nx, ny, "f64", w).set("algo", algo).set("int_path", int_path)
        if algo == "stream":
            p.set("depth", 4)
        src, dst = p.to_device(u0), p.empty()
        p.run(src, dst, steps)
        p.sync()
        refs.append(p.to_host(dst))
        p.close()
    assert np.array_equal(refs[0], refs[1])


def test_bad_depth_and_fallbacks():
    w = synth.weights(550)
    p = j2d5pt.Plan(100, 80, "f32", w).set("algo", "stream").set("depth", 5)
    a, b = p.empty(), p.empty()
    with pytest.raises(j2d5pt.J2DError) as e:
        p.run(a, b, 10)
    assert e.value.status == j2d5pt.J2D_ERR_ARG
    p.close()
    # adjoint runs of a stream plan take the tiles: still the one-step adjoint's values
    lam = synth.field(100, 80, 551)
    p = j2d5pt.Plan(100, 80, "f64", w).set("algo", "stream").set("depth", 4)
    q = j2d5pt.Plan(100, 80, "f64", w).set("algo", "onestep")
    outs = []
    for plan in (p, q):
        src, dst = plan.to_device(lam), plan.empty()
        plan.run_adjoint(src, dst, 6)
        plan.sync()
        outs.append(plan.to_host(dst))
    assert np.all(outs[0] == outs[1])
    desc = p.describe()
    assert "algo=stream" in desc, desc
