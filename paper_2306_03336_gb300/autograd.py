"""torch.autograd wrapper: u_T = M(w)^steps u_0, differentiable in u_0 and w.

The forward runs the library's kernels; the backward runs its adjoint and
weight-gradient kernels (the paper has no adjoint: this is the transpose of
its update, Section 3.1, Listing 1):

- lam_T = dL/du_T;  lam_t = M^T lam_{t+1}  (j2d5pt_run_adjoint);
- dL/du_0 = lam_0;
- dL/dw_d = sum_t sum_i lam_{t+1}[i] u_t[nbr_d(i)]  (j2d5pt_weight_grad; in the
  backward sweep fused with the adjoint step: j2d5pt_adjoint_step_wgrad).

The map is linear in u for fixed weights, so dL/du_0 needs no forward states
and is one adjoint run.  The weight gradient needs every u_t: the forward keeps
a checkpoint every `checkpoint` steps, and the backward recomputes one
segment at a time from its checkpoint, every state of it kept by one
state-keeping run (j2d5pt_run_states), and walks it in reverse.  Memory: steps/checkpoint + checkpoint grid copies
instead of steps.

Layout plumbing (copies between dense (ny+2, nx+2) tensors and the plan's
padded layout) uses torch; every arithmetic step runs in the CUDA library.
"""
import numpy as np
import torch

from . import j2d5pt


class J2D5PT:
    """A differentiable j2d5pt operator on one nx x ny grid (ring included in
    the (ny+2, nx+2) tensors it takes and returns)."""

    def __init__(self, nx, ny, dtype="f64", checkpoint=50):
        if checkpoint < 1:
            raise ValueError("checkpoint must be >= 1")
        self.nx, self.ny, self.dtype, self.checkpoint = int(nx), int(ny), dtype, int(checkpoint)
        self.plan = j2d5pt.Plan(nx, ny, dtype, np.full(5, 0.2))
        self._pool = []
        self._states = None

    def close(self):
        self.plan.close()
        self._pool = []
        self._states = None

    @property
    def torch_dtype(self):
        return self.plan.torch_dtype

    def _buf(self, i):
        while len(self._pool) <= i:
            self._pool.append(self.plan.empty())
        return self._pool[i]

    def _segment_states(self):
        # states 1 .. checkpoint-1 of a segment, one contiguous buffer
        if self._states is None and self.checkpoint > 1:
            self._states = self.plan.empty_states(self.checkpoint - 1)
        return self._states

    def _set_weights(self, w):
        self.plan.set_weights(w.detach().to("cpu", torch.float64).numpy())

    def _load(self, dense, buf):
        self.plan.view(buf).copy_(dense)
        return buf

    def __call__(self, u0, weights, steps):
        return _J2D5PTFn.apply(u0, weights, self, int(steps))


class _J2D5PTFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, w, op, steps):
        if u0.shape != (op.ny + 2, op.nx + 2) or u0.dtype != op.torch_dtype or not u0.is_cuda:
            raise ValueError("u0 must be a CUDA (ny+2, nx+2) tensor of the operator's dtype")
        if w.shape != (5,):
            raise ValueError("weights must have shape (5,)")
        op._set_weights(w)
        plan, c = op.plan, op.checkpoint
        nseg = (steps + c - 1) // c if steps > 0 else 0
        # checkpoints: the state at the start of every segment
        cks = [plan.empty() for _ in range(nseg)]
        cur = op._load(u0, cks[0] if nseg else op._buf(0))
        for j in range(nseg):
            n = min(c, steps - j * c)
            nxt = cks[j + 1] if j + 1 < nseg else op._buf(0)
            plan.run(cur, nxt, n)
            cur = nxt
        plan.sync()
        ctx.op, ctx.steps, ctx.cks = op, steps, cks
        return plan.view(cur).clone()

    @staticmethod
    def backward(ctx, g):
        op, steps, cks = ctx.op, ctx.steps, ctx.cks
        plan, c = op.plan, op.checkpoint
        lam = op._load(g.to(op.torch_dtype).contiguous(), op._buf(1))
        tmp = op._buf(2)
        dw = None
        if steps == 0:
            pass
        elif ctx.needs_input_grad[1]:
            dw = torch.zeros(5, dtype=torch.float64, device=g.device)
            nseg = len(cks)
            for j in reversed(range(nseg)):
                n = min(c, steps - j * c)
                # recompute this segment's states u_{jc} .. u_{jc+n-1} in one run
                states = [cks[j]]
                if n > 1:
                    buf = op._segment_states()
                    plan.run_states(cks[j], buf[:n - 1], n - 1)
                    states += [buf[i] for i in range(n - 1)]
                for t in reversed(range(n)):
                    # lam holds lam_{t+1}: one pass gives lam_t and the step's dL/dw
                    plan.adjoint_step_wgrad(states[t], lam, tmp, dw)
                    lam, tmp = tmp, lam
        else:
            plan.run_adjoint(lam, tmp, steps)
            lam = tmp
        plan.sync()
        grad_u0 = plan.view(lam).clone() if ctx.needs_input_grad[0] else None
        grad_w = dw.to(dtype=torch.float64) if dw is not None else None
        return grad_u0, grad_w, None, None


def j2d5pt_apply(u0, weights, steps, checkpoint=50, op=None):
    """Differentiable u_T = M(w)^steps u_0 for a dense (ny+2, nx+2) CUDA tensor."""
    if op is None:
        op = J2D5PT(u0.shape[1] - 2, u0.shape[0] - 2, "f64" if u0.dtype == torch.float64 else "f32", checkpoint)
    return op(u0, weights, steps)
