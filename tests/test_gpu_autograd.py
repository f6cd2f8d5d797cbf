"""Differentiation: the autograd wrapper's gradients against the oracle and
finite differences.

- small grids: dL/du0 and dL/dw against the oracle's full-trajectory reverse
  sweep (the literal transpose), <= 1e-12 relative;
- finite differences (central, h = 1e-6) on cells of u0 and on each weight;
- the full workload (4096^2 FP64, 500 steps, checkpoints every 50): dL/du0 at
  seeded cells against finite differences (tolerance from the rounding of L,
  about eps*|L|/h relative to the gradient) and against the oracle evaluated
  cell by cell: lam_0[i] = <M^T e_i, g>, the forward oracle run on the unit
  impulse at i over the window the impulse can reach in T steps.
"""
import numpy as np
import pytest

import oracle
from paper_2306_03336_gb300 import synth
from tests.gpu_util import TOL_F64

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


def _grads(u0, w, g, steps, checkpoint, need_w=True):
    import torch
    from paper_2306_03336_gb300.autograd import J2D5PT
    op = J2D5PT(u0.shape[1] - 2, u0.shape[0] - 2, "f64", checkpoint)
    ut = torch.tensor(u0, device="cuda", requires_grad=True)
    wt = torch.tensor(w, device="cuda", requires_grad=need_w)
    out = op(ut, wt, steps)
    loss = (out * torch.tensor(g, device="cuda")).sum()
    loss.backward()
    res = (ut.grad.cpu().numpy(), wt.grad.cpu().numpy() if need_w else None, out.detach().cpu().numpy())
    op.close()
    return res


@pytest.mark.parametrize("nx,ny,steps,ck", [(40, 30, 23, 5), (65, 17, 12, 50), (1, 1, 4, 3), (130, 90, 31, 8)])
def test_gradients_match_oracle_reverse_sweep(nx, ny, steps, ck):
    u0 = synth.field(nx, ny, 301 + nx)
    w = synth.weights(302)
    g = synth.field(nx, ny, 303 + ny)
    gu, gw, out = _grads(u0, w, g, steps, ck)
    lam0, dw = oracle.grad(u0, w, g, steps)
    assert np.abs(out - oracle.run(u0, w, steps)).max() <= TOL_F64
    assert np.abs(gu - lam0).max() <= TOL_F64 * np.abs(lam0).max()
    assert np.abs(gw - dw).max() <= TOL_F64 * np.abs(dw).max()
    gu2, _, _ = _grads(u0, w, g, steps, ck, need_w=False)  # pure adjoint path
    assert np.abs(gu2 - lam0).max() <= TOL_F64 * np.abs(lam0).max()


def test_finite_differences_medium():
    import torch
    from paper_2306_03336_gb300.autograd import J2D5PT
    nx, ny, steps = 256, 200, 60
    u0 = synth.field(nx, ny, 311)
    w = synth.weights(312)
    g = synth.field(nx, ny, 313)
    gu, gw, _ = _grads(u0, w, g, steps, 16)
    op = J2D5PT(nx, ny, "f64", 16)
    G = torch.tensor(g, device="cuda")

    def L(u, ww):
        with torch.no_grad():
            return float((op(torch.tensor(u, device="cuda"), torch.tensor(ww, device="cuda"), steps) * G).sum())
    h = 1e-6
    for (y, x) in synth.unit_cells(nx, ny, 5, 314):
        up, um = u0.copy(), u0.copy()
        up[y, x] += h
        um[y, x] -= h
        fd = (L(up, w) - L(um, w)) / (2 * h)
        assert abs(fd - gu[y, x]) <= 1e-4 * max(abs(gu[y, x]), 1e-3)
    for d in range(5):
        wp, wm = w.copy(), w.copy()
        wp[d] += h
        wm[d] -= h
        fd = (L(u0, wp) - L(u0, wm)) / (2 * h)
        assert abs(fd - gw[d]) <= 1e-4 * abs(gw[d])
    op.close()


def _oracle_lam0_at(g, w, steps, y, x):
    """lam_0[y, x] = <M^T e_(y,x), g>: forward oracle on the impulse, windowed to
    the cells it can reach (radius steps+1; outside them it stays zero)."""
    H, W = g.shape
    r = steps + 1
    y0, y1 = max(0, y - r), min(H - 1, y + r)
    x0, x1 = max(0, x - r), min(W - 1, x + r)
    e = np.zeros((y1 - y0 + 1, x1 - x0 + 1))
    e[y - y0, x - x0] = 1.0
    out = oracle.run(e, w, steps, threads=oracle.max_threads())
    return oracle.dot(out, np.ascontiguousarray(g[y0:y1 + 1, x0:x1 + 1]))


def test_full_workload_4096_500_steps_checkpoint_50():
    import torch
    from paper_2306_03336_gb300.autograd import J2D5PT
    cfg = synth.WORKLOADS["j2d5pt_f64_4096x4096_500_adjoint"]
    nx, ny, steps, ck = cfg["nx"], cfg["ny"], cfg["steps"], cfg["checkpoint"]
    u0 = synth.field(nx, ny, synth.data_seed(cfg["index"]))
    w = synth.weights(synth.weight_seed(cfg["index"]))
    g = synth.field(nx, ny, synth.data_seed(cfg["index"]) + 7)
    op = J2D5PT(nx, ny, "f64", ck)
    ut = torch.tensor(u0, device="cuda", requires_grad=True)
    wt = torch.tensor(w, device="cuda", requires_grad=True)
    G = torch.tensor(g, device="cuda")
    (op(ut, wt, steps) * G).sum().backward()
    gu = ut.grad.cpu().numpy()
    gw = wt.grad.cpu().numpy()
    cells = synth.unit_cells(nx, ny, 20, synth.data_seed(cfg["index"]) + 8)
    # CPU oracle, cell by cell (5 of the 20 cells: each is a 1003^2 x 500-step oracle run)
    for (y, x) in cells[:5]:
        ref = _oracle_lam0_at(g, w, steps, y, x)
        assert abs(gu[y, x] - ref) <= TOL_F64 * abs(ref)
    # central finite differences on all 20 cells; L is linear in u0, so the only
    # error is the rounding of L: about eps * |L| / h
    with torch.no_grad():
        base = op(torch.tensor(u0, device="cuda"), wt.detach(), steps)
        Lmag = float((base * G).abs().sum())
    h = 1e-6
    tol = 8 * 2.0 ** -53 * Lmag / h
    for (y, x) in cells:
        vals = []
        for s in (+1, -1):
            u = u0.copy()
            u[y, x] += s * h
            with torch.no_grad():
                vals.append(float((op(torch.tensor(u, device="cuda"), wt.detach(), steps) * G).sum()))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(fd - gu[y, x]) <= tol + 1e-2 * abs(gu[y, x])
    # weight gradient: Euler's identity needs a zero ring; check finite differences instead
    for d in range(5):
        vals = []
        for s in (+1, -1):
            ww = w.copy()
            ww[d] += s * 1e-7
            with torch.no_grad():
                vals.append(float((op(torch.tensor(u0, device="cuda"), torch.tensor(ww, device="cuda"), steps) * G).sum()))
        fd = (vals[0] - vals[1]) / 2e-7
        assert abs(fd - gw[d]) <= 1e-4 * abs(gw[d])
    op.close()
