"""The second stencil shape, the 3x3 box (j2d9pt), through the one-step
kernel and the skewed serial tiles: against the box oracle, bit for bit
between the kernels, bit for bit against an exact rational model of the FP64
cell arithmetic (the nine-term FMA chain and the correctly rounded nine-term
sum of the integer path), and at 16384^2 with the benchmark's launch
configuration."""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from paper_2306_03336_gb300 import j2d5pt, synth
from tests.gpu_util import TOL_F64, blocks_for, rel_err, window_block

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


box_weights = synth.box_weights


W_DYADIC = np.array([1, 1, 2, 2, 3, 2, 1, 3, 1], dtype=np.float64) / 16


def f32_box_bound(steps):
    """Binary32 storage and arithmetic against the FP64 oracle, values in
    [0, 1) and positive weights summing to 1: input rounding, weight rounding
    (nine weights) and up to ten roundings per step, accumulated linearly."""
    return (1 + 20 * max(steps, 1)) * 2.0 ** -24


def gpu_box(u0, w, steps, dtype="f64", algo="onestep", depth=None, wx=None, alias=False, int_path=None):
    ny, nx = u0.shape[0] - 2, u0.shape[1] - 2
    p = j2d5pt.Plan.box9(nx, ny, dtype, w).set("algo", algo)
    if depth:
        p.set("depth", depth)
    if wx:
        p.set("tile_wx", wx)
    if int_path is not None:
        p.set("int_path", int_path)
    src = p.to_device(u0 if dtype == "f64" else u0.astype(np.float32))
    dst = src if alias else p.empty()
    p.run(src, dst, steps)
    p.sync()
    out = p.to_host(dst)
    p.close()
    return out


SIZES = [(1, 1), (1, 7), (7, 1), (5, 3), (63, 65), (130, 67), (257, 300)]


@pytest.mark.parametrize("algo", ["onestep", "skewed", "stream"])
@pytest.mark.parametrize("nx,ny", SIZES)
def test_box_against_oracle_and_ring(algo, nx, ny):
    u0 = synth.field(nx, ny, 900 + nx + 7 * ny)
    w = box_weights(901 + nx)
    for steps in (0, 1, 2, 7):
        ref = oracle.box_run(u0, w, steps)
        got = gpu_box(u0, w, steps, algo=algo, depth=3)
        assert rel_err(got, ref) <= TOL_F64, (nx, ny, steps)
        for sl in (np.s_[0, :], np.s_[-1, :], np.s_[:, 0], np.s_[:, -1]):
            assert np.array_equal(got[sl], u0[sl])


@pytest.mark.parametrize("algo", ["onestep", "skewed", "stream"])
def test_box_dyadic_bit_identical(algo):
    nx, ny = 100, 37
    u0 = synth.dyadic_field(nx, ny, 905)
    assert np.array_equal(gpu_box(u0, W_DYADIC, 6, algo=algo, depth=4), oracle.box_run(u0, W_DYADIC, 6))


@pytest.mark.parametrize("algo", ["onestep", "skewed", "stream"])
def test_box_in_place_alias(algo):
    nx, ny = 150, 90
    u0 = synth.field(nx, ny, 906)
    w = box_weights(907)
    for steps in (1, 4, 5):
        assert rel_err(gpu_box(u0, w, steps, algo=algo, depth=3, alias=True), oracle.box_run(u0, w, steps)) <= TOL_F64


SKEW = [(1, 2), (2, 4), (3, 8), (5, 1), (8, 4), (13, 2), (4, 16)]


@pytest.mark.parametrize("depth,wx", SKEW)
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_box_skewed_bitwise_equal_to_onestep(depth, wx, dtype):
    nx, ny, steps = 700, 450, 13
    u0 = synth.field(nx, ny, 910)
    w = box_weights(911)
    if dtype == "f32":
        u0 = u0.astype(np.float32)
    ref = gpu_box(u0, w, steps, dtype=dtype, algo="onestep")
    got = gpu_box(u0, w, steps, dtype=dtype, algo="skewed", depth=depth, wx=wx)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("dtype,depth", [("f64", 2), ("f64", 3), ("f64", 4), ("f32", 4), ("f32", 6), ("f32", 8)])
@pytest.mark.parametrize("nx,ny", [(700, 450), (1, 1), (5, 3), (3, 400), (129, 257)])
def test_box_stream_bitwise_equal_to_onestep(dtype, depth, nx, ny):
    """The stream schedule on the box: every depth it has a kernel for, step
    counts below, at and across whole passes, in place and not."""
    u0 = synth.field(nx, ny, 915 + nx)
    w = box_weights(916)
    if dtype == "f32":
        u0 = u0.astype(np.float32)
    for steps in sorted({1, depth - 1, depth, 2 * depth + 1, 13}):
        if steps < 1:
            continue
        ref = gpu_box(u0, w, steps, dtype=dtype, algo="onestep")
        assert np.array_equal(gpu_box(u0, w, steps, dtype=dtype, algo="stream", depth=depth), ref), (steps,)
        assert np.array_equal(gpu_box(u0, w, steps, dtype=dtype, algo="stream", depth=depth, alias=True), ref)


@pytest.mark.parametrize("algo", ["onestep", "skewed", "stream"])
def test_box_f32_against_f32_and_f64_oracles(algo):
    nx, ny, steps = 333, 211, 40
    u0 = synth.field(nx, ny, 920)
    w = box_weights(921)
    got = gpu_box(u0.astype(np.float32), w, steps, dtype="f32", algo=algo, depth=8)
    u32 = u0.astype(np.float32).astype(np.float64)
    assert rel_err(got, oracle.box_run(u32, w, steps)) <= f32_box_bound(steps)
    assert rel_err(got, oracle.box_run_f32(u0, w, steps).astype(np.float64)) <= f32_box_bound(steps)


def test_box_forward_only_calls_refused():
    import torch
    p = j2d5pt.Plan.box9(64, 64, "f64", box_weights(930))
    a, b = p.empty(), p.empty()
    dw = torch.zeros(5, dtype=torch.float64, device="cuda")
    for call in (lambda: p.run_adjoint(a, b, 1), lambda: p.weight_grad(a, b, dw),
                 lambda: p.adjoint_step_wgrad(a, b, p.empty(), dw), lambda: p.set_weights(np.full(5, 0.2))):
        with pytest.raises(j2d5pt.J2DError) as e:
            call()
        assert e.value.status == j2d5pt.J2D_ERR_UNSUPPORTED
    assert "stencil=box9" in p.describe()
    p.close()


def test_box_autotune(monkeypatch):
    import torch
    monkeypatch.delenv("J2D_TUNE_CACHE", raising=False)
    nx, ny, steps = 900, 700, 48
    u0 = synth.field(nx, ny, 940)
    w = box_weights(941)
    p = j2d5pt.Plan.box9(nx, ny, "f64", w)
    src, dst = p.to_device(u0), p.empty()
    desc = p.autotune(src, dst, steps)
    assert "algo=onestep" in desc or "algo=skewed" in desc or "algo=stream" in desc
    dst.zero_()
    p.run(src, dst, steps)
    p.sync()
    assert rel_err(p.to_host(dst), oracle.box_run(u0, w, steps, threads=oracle.max_threads())) <= TOL_F64
    q = j2d5pt.Plan.box9(nx, ny, "f64", w).set("algo", "onestep")
    ref = q.empty()
    q.run(src, ref, steps)
    q.sync()
    assert torch.equal(p.view(dst), q.view(ref))
    p.close()
    q.close()


# ---- exact rational model of the FP64 box cell ------------------------------

def _biased_exp(v):
    return int((np.float64(v).view(np.uint64) >> np.uint64(52)) & np.uint64(0x7FF))


def _pos_normal(v):
    return v > 0 and 1 <= _biased_exp(v) <= 2046


CHAIN = (1, 0, 2, 4, 3, 5, 7, 6, 8)  # user index of each term of the FMA chain


def model_box_cell(w, vals, x, y, mask, guard):
    """w and vals in the user's order (rows y-1, y, y+1; columns x-1, x, x+1)."""
    if (mask >> (((y & 3) << 1) | (x & 1))) & 1 and all(_pos_normal(a) for a in w) \
            and all(_pos_normal(v) for v in vals):
        E = [_biased_exp(a) + _biased_exp(v) for a, v in zip(w, vals)]
        if max(E) - min(E) <= guard:
            r = float(sum(Fraction(a) * Fraction(v) for a, v in zip(w, vals)))
            if 1 <= _biased_exp(r) <= 2046:
                return r
    i0 = CHAIN[0]
    r = float(Fraction(w[i0]) * Fraction(vals[i0]))
    for i in CHAIN[1:]:
        r = float(Fraction(w[i]) * Fraction(vals[i]) + Fraction(r))
    return r


def model_box_step(u, w, mask, guard):
    ny, nx = u.shape[0] - 2, u.shape[1] - 2
    out = u.copy()
    for y in range(1, ny + 1):
        for x in range(1, nx + 1):
            vals = [float(u[y + dy, x + dx]) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
            out[y, x] = model_box_cell([float(a) for a in w], vals, x, y, mask, guard)
    return out


def _fields(nx, ny):
    rng = np.random.Generator(np.random.PCG64(2306033397))
    shape = (ny + 2, nx + 2)
    k = rng.integers(1, 31, size=shape)
    short = (1.0 + np.floor(rng.random(shape) * 2.0 ** k) / 2.0 ** k) * 2.0 ** rng.integers(-6, 1, size=shape) / 2
    spread = synth.field(nx, ny, 951) * 2.0 ** -rng.integers(0, 40, size=shape)
    mixed = synth.field(nx, ny, 952) - 0.25
    mixed[rng.random(shape) < 0.05] = 0.0
    return {"uniform": synth.field(nx, ny, 950), "short": short, "spread": spread, "mixed": mixed}


@pytest.mark.parametrize("int_path", [1, 0])
@pytest.mark.parametrize("fname", ["uniform", "short", "spread", "mixed"])
def test_box_cells_bit_exact(fname, int_path):
    nx, ny, steps = 70, 45, 3
    mask, guard = j2d5pt.j2d5pt_arith_info()
    mask = mask if int_path else 0
    u0 = _fields(nx, ny)[fname]
    w = box_weights(960)
    ref = u0
    for _ in range(steps):
        ref = model_box_step(ref, w, mask, guard)
    for algo in ("onestep", "skewed", "stream"):
        got = gpu_box(u0, w, steps, algo=algo, depth=steps, int_path=int_path)
        bad = np.argwhere(got != ref)
        assert bad.size == 0, "%s/%s/int_path=%d: %d cells differ, first %s" % (algo, fname, int_path, len(bad),
                                                                                 tuple(bad[0]))


def test_box_integer_path_is_used():
    mask, guard = j2d5pt.j2d5pt_arith_info()
    u0 = _fields(40, 30)["uniform"]
    w = box_weights(961)
    exact = model_box_step(u0, w, mask, guard)
    chain = model_box_step(u0, w, 0, guard)
    assert np.count_nonzero(exact != chain) > 0.05 * 40 * 30 * bin(mask).count("1") / 8
    assert j2d5pt.j2d9pt_measure_exact_rate() > 1e9


# ---- full size, the benchmark's configuration ------------------------------------

@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_box_16384_full_grid(dtype):
    import torch
    n, steps = 16384, 1000
    u0 = synth.field(n, n, synth.data_seed(1))
    w = box_weights(synth.weight_seed(1))
    uin = u0 if dtype == "f64" else u0.astype(np.float32)
    ref_plan = j2d5pt.Plan.box9(n, n, dtype, w).set("algo", "onestep")
    src = ref_plan.to_device(uin)
    ref = ref_plan.empty()
    ref_plan.run(src, ref, steps)
    ref_plan.sync()
    ref_plan.close()
    p = j2d5pt.Plan.box9(n, n, dtype, w)
    dst = p.empty()
    p.autotune(src, dst, steps)
    dst.zero_()
    p.run(src, dst, steps)
    p.sync()
    assert torch.equal(p.view(dst), p.view(ref)), p.describe()
    u64 = u0 if dtype == "f64" else u0.astype(np.float32).astype(np.float64)
    tol = TOL_F64 if dtype == "f64" else f32_box_bound(steps)
    v = p.view(dst)
    for (y0, y1, x0, x1) in blocks_for(n, n, size=200)[:3]:
        e = window_block(oracle, u64, w, steps, y0, y1, x0, x1, box=True)
        got = v[y0:y1, x0:x1].double().cpu().numpy()
        assert (np.abs(got - e) / np.maximum(np.abs(e), 1e-300)).max() <= tol, (p.describe(), y0, x0)
    p.close()
