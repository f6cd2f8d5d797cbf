"""The state-keeping forward run (j2d5pt_run_states): every intermediate
state, ring included, bit for bit equal to chained single-step runs of the
one-step kernel, for every algorithm (the skewed and two-step FP32
schedules run as single-step tiles there; the stream schedule stores every
step from its pipeline, also at depths without a state-keeping kernel of
their own, which take the default depth), ragged sizes, depths that do and
do not divide the step count; the oracle on one case; argument errors."""
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


def _chained(nx, ny, dtype, w, u0, steps):
    """States 1..steps by single steps of the one-step kernel (logical views, on the host)."""
    p = j2d5pt.Plan(nx, ny, dtype, w).set("algo", "onestep")
    cur = p.to_device(u0)
    out = []
    for _ in range(steps):
        nxt = p.empty()
        p.run(cur, nxt, 1)
        out.append(p.to_host(nxt))
        cur = nxt
    p.close()
    return out


def _states(nx, ny, dtype, w, u0, steps, algo, depth, wx):
    p = j2d5pt.Plan(nx, ny, dtype, w)
    if algo != "auto":
        p.set("algo", algo)
    if depth:
        p.set("depth", depth)
    if wx:
        p.set("tile_wx", wx)
    src = p.to_device(u0)
    st = p.empty_states(steps)
    p.run_states(src, st, steps)
    p.sync()
    got = [p.to_host(st[t]) for t in range(steps)]
    p.close()
    return got


CONFIGS = [("onestep", 0, 0), ("tiles", 1, 2), ("tiles", 3, 4), ("tiles", 4, 1), ("tiles", 7, 8), ("bands", 3, 0),
           ("resident", 0, 0), ("skewed", 4, 4), ("stream", 2, 0), ("stream", 3, 0), ("stream", 4, 0),
           ("stream", 6, 0), ("auto", 0, 0)]


@pytest.mark.parametrize("algo,depth,wx", CONFIGS)
@pytest.mark.parametrize("nx,ny", [(300, 200), (1, 1), (129, 77), (64, 64), (257, 3)])
def test_states_bitwise_f64(algo, depth, wx, nx, ny):
    w = synth.weights(701)
    u0 = synth.field(nx, ny, 702 + nx)
    steps = 13
    ref = _chained(nx, ny, "f64", w, u0, steps)
    got = _states(nx, ny, "f64", w, u0, steps, algo, depth, wx)
    for t in range(steps):
        assert np.array_equal(got[t], ref[t]), (algo, depth, wx, nx, ny, t + 1)


@pytest.mark.parametrize("algo,depth,wx", [("tiles", 8, 2), ("tiles", 3, 4), ("bands", 5, 0), ("resident", 0, 0),
                                           ("skewed", 8, 4), ("stream", 4, 0), ("stream", 8, 0), ("stream", 12, 0)])
@pytest.mark.parametrize("nx,ny", [(300, 200), (513, 31), (7, 9)])
def test_states_bitwise_f32(algo, depth, wx, nx, ny):
    # FP32 tiles would sweep two steps per pass; a state-keeping run takes one
    w = synth.weights(711)
    u0 = synth.field(nx, ny, 712, dtype=np.float32)
    steps = 10
    ref = _chained(nx, ny, "f32", w, u0, steps)
    got = _states(nx, ny, "f32", w, u0, steps, algo, depth, wx)
    for t in range(steps):
        assert np.array_equal(got[t], ref[t]), (algo, nx, ny, t + 1)


@pytest.mark.parametrize("steps", [1, 2, 4, 5])
def test_states_short_runs_and_oracle(steps):
    nx, ny = 190, 170
    w = synth.weights(721)
    u0 = synth.field(nx, ny, 722)
    got = _states(nx, ny, "f64", w, u0, steps, "tiles", 4, 2)
    for t in range(steps):
        assert rel_err(got[t], oracle.run(u0, w, t + 1)) <= TOL_F64


def test_states_argument_errors():
    import torch
    nx, ny = 64, 48
    w = synth.weights(731)
    p = j2d5pt.Plan(nx, ny, "f64", w)
    src = p.to_device(synth.field(nx, ny, 732))
    st = p.empty_states(4)
    for bad_steps in (0, -1):
        with pytest.raises(j2d5pt.J2DError) as e:
            p.run_states(src, st, bad_steps)
        assert e.value.status == j2d5pt.J2D_ERR_ARG
    with pytest.raises(j2d5pt.J2DError) as e:  # input inside the state buffer
        p.run_states(st[1], st, 4)
    assert e.value.status == j2d5pt.J2D_ERR_ARG
    flat = torch.zeros(st.numel() + 2, dtype=torch.float64, device="cuda")
    with pytest.raises(j2d5pt.J2DError) as e:  # 8-byte offset: not 16-byte aligned
        p.run_states(src, flat[1:], 2)
    assert e.value.status == j2d5pt.J2D_ERR_ALIGN
    p.close()
    box = j2d5pt.Plan.box9(nx, ny, "f64", synth.box_weights(733))
    with pytest.raises(j2d5pt.J2DError) as e:
        box.run_states(box.to_device(synth.field(nx, ny, 734)), box.empty_states(2), 2)
    assert e.value.status == j2d5pt.J2D_ERR_UNSUPPORTED
    box.close()
    b = j2d5pt.Plan.batch([(32, 32), (40, 20)], "f64", np.stack([w, w]))
    with pytest.raises(j2d5pt.J2DError) as e:
        j2d5pt.j2d5pt_run_states(b.handle, b.empty(0), b.empty(0), 2)
    assert e.value.status == j2d5pt.J2D_ERR_ARG
    b.close()
