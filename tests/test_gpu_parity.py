"""GPU parity: every kernel family against the CPU oracle on seeded inputs.

Bars: FP64 within 1e-12 max relative error of the oracle; dyadic inputs and
weights (exact in floating point) bit-identical to the oracle; the ring held
exactly; all kernel families bit-identical to the one-step kernel for the same
inputs (same operand order), which pins the temporally blocked paths to the
one-step path for every tile shape and depth.
"""
import numpy as np
import pytest

import oracle
from paper_2306_03336_gb300 import j2d5pt, synth
from tests.gpu_util import TOL_F64, cell_rel_err, f32_bound, rel_err

pytestmark = pytest.mark.gpu

ALGOS = ["onestep", "resident", "bands", "tiles", "skewed", "stream"]
DEPTH = {"bands": 3, "tiles": 3, "skewed": 3}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def gpu_run(u0, w, steps, dtype="f64", algo="onestep", depth=None, wx=None, alias=False, adjoint=False):
    ny, nx = u0.shape[0] - 2, u0.shape[1] - 2
    p = j2d5pt.Plan(nx, ny, dtype, w)
    p.set("algo", algo)
    if depth is None:
        depth = DEPTH.get(algo)
    if depth is not None:
        p.set("depth", depth)
    if wx is not None:
        p.set("tile_wx", wx)
    src = p.to_device(u0)
    dst = src if alias else p.empty()
    if adjoint:
        p.run_adjoint(src, dst, steps)
    else:
        p.run(src, dst, steps)
    p.sync()
    out = p.to_host(dst)
    p.close()
    return out


@pytest.mark.parametrize("algo", ALGOS)
def test_config_512_f64_16_steps(algo):
    nx = ny = 512
    u0 = synth.field(nx, ny, synth.data_seed(0))
    w = synth.weights(synth.weight_seed(0))
    ref = oracle.run(u0, w, 16, threads=4)
    got = gpu_run(u0, w, 16, algo=algo)
    assert rel_err(got, ref) <= TOL_F64
    assert cell_rel_err(got, ref) <= TOL_F64


SIZES = [(1, 1), (1, 7), (7, 1), (5, 3), (63, 65), (130, 67), (257, 300)]


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("nx,ny", SIZES)
def test_ragged_sizes_and_ring(algo, nx, ny):
    u0 = synth.field(nx, ny, 100 + nx + 7 * ny)
    w = synth.weights(200 + nx)
    for steps in (0, 1, 2, 7):
        ref = oracle.run(u0, w, steps)
        got = gpu_run(u0, w, steps, algo=algo)
        assert rel_err(got, ref) <= TOL_F64, (nx, ny, steps)
        for sl in (np.s_[0, :], np.s_[-1, :], np.s_[:, 0], np.s_[:, -1]):
            assert np.array_equal(got[sl], u0[sl])


@pytest.mark.parametrize("algo", ALGOS)
def test_dyadic_inputs_bit_identical(algo):
    nx, ny = 100, 37
    w = synth.dyadic_weights()
    u0 = synth.dyadic_field(nx, ny, 5)
    ref = oracle.run(u0, w, 6)
    got = gpu_run(u0, w, 6, algo=algo)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("algo", ALGOS)
def test_in_place_alias(algo):
    nx, ny = 150, 90
    u0 = synth.field(nx, ny, 9)
    w = synth.weights(10)
    for steps in (1, 4, 5):
        ref = oracle.run(u0, w, steps)
        assert rel_err(gpu_run(u0, w, steps, algo=algo, alias=True), ref) <= TOL_F64


@pytest.mark.parametrize("algo", ALGOS)
def test_f32_against_f32_and_f64_oracles(algo):
    nx, ny, steps = 333, 211, 40
    u0 = synth.field(nx, ny, 31)
    w = synth.weights(32)
    got = gpu_run(u0.astype(np.float32), w, steps, dtype="f32", algo=algo)
    ref64 = oracle.run(u0.astype(np.float32).astype(np.float64), w, steps)
    assert rel_err(got, ref64) <= f32_bound(steps)
    ref32 = oracle.run_f32(u0, w, steps).astype(np.float64)
    assert rel_err(got, ref32) <= f32_bound(steps)
    # dyadic data and weights are exact in binary32 for 4 steps
    wd = synth.dyadic_weights()
    ud = synth.dyadic_field(nx, ny, 33)
    assert np.array_equal(gpu_run(ud, wd, 4, dtype="f32", algo=algo), oracle.run(ud, wd, 4))


def test_adjoint_onestep_against_oracle():
    nx, ny, steps = 141, 77, 9
    lam = synth.field(nx, ny, 41)
    w = synth.weights(42)
    ref = oracle.adjoint_run(lam, w, steps)
    p = j2d5pt.Plan(nx, ny, "f64", w).set("algo", "onestep")
    src = p.to_device(lam)
    dst = p.empty()
    p.run_adjoint(src, dst, steps)
    p.sync()
    assert rel_err(p.to_host(dst), ref) <= TOL_F64
    # dyadic: bit-identical, ring accumulation included
    wd = synth.dyadic_weights()
    ld = synth.dyadic_field(nx, ny, 43)
    p2 = j2d5pt.Plan(nx, ny, "f64", wd).set("algo", "onestep")
    src = p2.to_device(ld)
    p2.run_adjoint(src, dst := p2.empty(), 5)
    p2.sync()
    assert np.array_equal(p2.to_host(dst), oracle.adjoint_run(ld, wd, 5))


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_weight_grad_against_oracle(dtype):
    import torch
    nx, ny = 517, 263
    u = synth.field(nx, ny, 51)
    lam = synth.field(nx, ny, 52)
    w = synth.weights(53)
    npd = np.float64 if dtype == "f64" else np.float32
    u_, lam_ = u.astype(npd).astype(np.float64), lam.astype(npd).astype(np.float64)
    ref = oracle.weight_grad(u_, lam_)
    p = j2d5pt.Plan(nx, ny, dtype, w)
    dw = torch.full((5,), 0.5, dtype=torch.float64, device="cuda")
    p.weight_grad(p.to_device(u), p.to_device(lam), dw)
    p.sync()
    got = dw.cpu().numpy() - 0.5
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    # reproducible: same order every call
    dw2 = torch.full((5,), 0.5, dtype=torch.float64, device="cuda")
    p.weight_grad(p.to_device(u), p.to_device(lam), dw2)
    assert torch.equal(dw, dw2)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("nx,ny", [(517, 263), (70, 45), (1, 1), (3, 700)])
def test_adjoint_step_wgrad_fused(dtype, nx, ny):
    """One pass: lam_t bit-identical to the one-step adjoint, dw equal to the
    separate reduction up to summation order and to the oracle within 1e-12."""
    import torch
    u = synth.field(nx, ny, 54)
    lam = synth.field(nx, ny, 55)
    w = synth.weights(56)
    npd = np.float64 if dtype == "f64" else np.float32
    u_, lam_ = u.astype(npd).astype(np.float64), lam.astype(npd).astype(np.float64)
    p = j2d5pt.Plan(nx, ny, dtype, w)
    U, L1 = p.to_device(u), p.to_device(lam)
    L0, L0b = p.empty(), p.empty()
    dw = torch.full((5,), 0.5, dtype=torch.float64, device="cuda")
    dw_sep = torch.full((5,), 0.5, dtype=torch.float64, device="cuda")
    p.adjoint_step_wgrad(U, L1, L0, dw)
    p.weight_grad(U, L1, dw_sep)
    p.run_adjoint(L1, L0b, 1)
    p.sync()
    assert np.array_equal(p.to_host(L0), p.to_host(L0b))
    ref = oracle.weight_grad(u_, lam_)
    got, sep = dw.cpu().numpy() - 0.5, dw_sep.cpu().numpy() - 0.5
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(got - sep).max() <= 1e-13 * np.abs(ref).max()
    if dtype == "f64":
        assert rel_err(p.to_host(L0), oracle.adjoint_step(lam, w)) <= TOL_F64
    with pytest.raises(j2d5pt.J2DError):
        p.adjoint_step_wgrad(U, L1, L1, dw)  # output aliases an input


def test_run_host_end_to_end_matches_device_run():
    nx, ny, steps = 300, 200, 11
    u0 = synth.field(nx, ny, 61)
    w = synth.weights(62)
    p = j2d5pt.Plan(nx, ny, "f64", w)
    host = p.run_host(u0, steps)
    dev = gpu_run(u0, w, steps)
    assert np.array_equal(host, dev)
    assert rel_err(host, oracle.run(u0, w, steps)) <= TOL_F64


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("nx,ny", [(300, 200), (1, 1), (7, 13), (1023, 5), (129, 257)])
@pytest.mark.parametrize("pinned", [True, False])
def test_run_host_pinned_and_pageable(dtype, nx, ny, pinned):
    """A pinned input is gathered on the device by a kernel, a pageable one
    copied; odd row lengths leave the host rows unaligned to 16 bytes.  Both
    give the device run's bits, and 0 steps give the input back."""
    import torch
    u0 = synth.field(nx, ny, 63 + nx).astype(np.float64 if dtype == "f64" else np.float32)
    w = synth.weights(64)
    p = j2d5pt.Plan(nx, ny, dtype, w)
    src = torch.from_numpy(u0).pin_memory().numpy() if pinned else u0.copy()
    out = torch.empty(u0.shape, dtype=p.torch_dtype).pin_memory().numpy() if pinned else None
    assert np.array_equal(p.run_host(src, 0, out=out), u0)
    host = p.run_host(src, 9, out=out).copy()
    d_in = p.to_device(u0)
    d_out = p.empty()
    p.run(d_in, d_out, 9)
    assert np.array_equal(host, p.to_host(d_out))
    p.close()


def test_argument_errors_on_device():
    import torch
    p = j2d5pt.Plan(64, 64, "f64", synth.weights(1))
    a = p.empty()
    b = p.empty()
    with pytest.raises(j2d5pt.J2DError) as e:
        p.run(a, b, -1)
    assert e.value.status == j2d5pt.J2D_ERR_ARG
    flat = torch.zeros(66 * 80 + 1, dtype=torch.float64, device="cuda")
    with pytest.raises(j2d5pt.J2DError) as e:
        j2d5pt.j2d5pt_run(p.handle, flat.data_ptr() + 8, b, 1)
    assert e.value.status == j2d5pt.J2D_ERR_ALIGN
    with pytest.raises(j2d5pt.J2DError):
        p.set("depth", 100000)
    p.close()


def test_fma_rate_probe():
    r64 = j2d5pt.j2d5pt_measure_fma_rate(j2d5pt.J2D_F64)
    r32 = j2d5pt.j2d5pt_measure_fma_rate(j2d5pt.J2D_F32)
    assert r64 > 1e10 and r32 > r64


INVARIANCE = [("resident", None, None), ("bands", 1, None), ("bands", 2, None), ("bands", 5, None),
              ("tiles", 1, 1), ("tiles", 2, 2), ("tiles", 4, 4), ("tiles", 6, 8), ("tiles", 3, 16),
              ("skewed", 1, 2), ("skewed", 2, 4), ("skewed", 5, 8), ("skewed", 3, 1), ("skewed", 4, 16),
              ("skewed", 13, 2), ("skewed", 8, 4)]


@pytest.mark.parametrize("algo,depth,wx", INVARIANCE)
@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_tiling_invariance_bitwise(algo, depth, wx, dtype):
    # same operand order in every kernel: any tiling / depth gives the one-step result bit for bit
    nx, ny, steps = 700, 450, 13
    u0 = synth.field(nx, ny, 71)
    w = synth.weights(72)
    if dtype == "f32":
        u0 = u0.astype(np.float32)
    ref = gpu_run(u0, w, steps, dtype=dtype, algo="onestep")
    got = gpu_run(u0, w, steps, dtype=dtype, algo=algo, depth=depth, wx=wx)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("nx,ny", [(1, 1), (5, 3), (130, 67), (257, 300)])
def test_adjoint_all_kernels(algo, nx, ny):
    lam = synth.field(nx, ny, 81 + nx)
    w = synth.weights(82)
    for steps in (1, 6):
        ref = oracle.adjoint_run(lam, w, steps)
        got = gpu_run(lam, w, steps, algo=algo, adjoint=True)
        assert rel_err(got, ref) <= TOL_F64, (nx, ny, steps)
        one = gpu_run(lam, w, steps, algo="onestep", adjoint=True)
        assert np.all(got == one)  # numerically identical (sign of zero aside)


def test_bounded_wait_reports_timeout_and_context_survives():
    # a strip whose step counter is never published (host-set fault injection):
    # its neighbours' waits run out after the plan's limit, the kernel finishes,
    # the status says J2D_ERR_TIMEOUT, and the next run on the same plan is correct
    nx, ny, steps = 2048, 512, 20
    u0 = synth.field(nx, ny, 91)
    w = synth.weights(92)
    p = j2d5pt.Plan(nx, ny, "f64", w).set("algo", "resident").set("timeout_ms", 100).set("fault_inject", 1)
    src = p.to_device(u0)
    dst = p.empty()
    p.run(src, dst, steps)
    with pytest.raises(j2d5pt.J2DError) as e:
        p.sync()
    assert e.value.status == j2d5pt.J2D_ERR_TIMEOUT
    p.set("fault_inject", 0)
    p.run(src, dst, steps)
    p.sync()
    assert rel_err(p.to_host(dst), oracle.run(u0, w, steps, threads=4)) <= TOL_F64
    p.close()
