"""Differentiable Householder Dice trajectories.

`trajectory(hd, x1, schedule, f, params)` runs the dynamics of eq. (dynamics),

    y_t = M_t x_t  (M_t = Q^T where schedule[t-1] is true, else Q; through the library),
    x_{t+1} = f(t, y_t, x_t, x_{t-1}, *params)   (the caller's f_t, plain torch ops),

on the state `hd` (reset to its seed first) and returns x_{T+1} as a tensor that autograd can
differentiate with respect to x_1 and `params`, with the Gaussian draws held fixed.

Backward walks the steps last to first.  For each t it differentiates the caller's f_t
locally (torch), which gives dLoss/dy_t and the f_t parts of dLoss/dx_t and dLoss/dx_{t-1}.
It then calls the library's reverse step (hd_adjoint_step, CUDA), which returns the part of
dLoss/dx_t that flows through y_t and through every later product that used the reflector
built from x_t.  x_{t-1} is None at t = 1.

A batched state (HDBatch, every trial of the same dimensions) runs all its trials at once:
vectors are packed, f_t sees the packed vectors, and every reverse step is one set of
launches for the whole batch.

Memory: without checkpointing the library records every x_t, and this module keeps every y_t.
With `checkpoint=S` only x_t at every S-th step is kept.  In backward, each segment is
recomputed from its first x with hd_probe_at: the representation as it stood after step s
maps x_s to y_s exactly on its revealed part (eq. H_t / eq. Gaussian_t), with the reflectors
that step used, so no step is redrawn.  The
segment's x_t are then passed back to the library.  Recomputed values agree with the forward
pass up to rounding; a discontinuous f_t can amplify that.
"""
import torch

from .binding import HD, HDBatch


class _Trajectory(torch.autograd.Function):
    @staticmethod
    def forward(ctx, hd, schedule, f, checkpoint, x1, *params):
        if not isinstance(hd, (HD, HDBatch)):
            raise TypeError("hd must be a paper_2101_07464_gb300.HD or HDBatch state")
        if isinstance(hd, HDBatch) and checkpoint is not None:
            raise ValueError("segment checkpointing needs hd_probe, which takes single-trial states")
        T = len(schedule)
        hd.reset()
        hd.adjoint_enable(record_x=checkpoint is None)
        x, xprev = x1.detach(), None
        xs, ys, marks = [], [], {}
        with torch.no_grad():
            for t in range(1, T + 1):
                if checkpoint is None:
                    xs.append(x)
                elif (t - 1) % checkpoint == 0:
                    marks[t] = (x, xprev)
                y = hd.apply(x, bool(schedule[t - 1]))
                if checkpoint is None:
                    ys.append(y)
                x, xprev = f(t, y, x, xprev, *params), x
        ctx.hd, ctx.schedule, ctx.f, ctx.checkpoint = hd, list(schedule), f, checkpoint
        ctx.xs, ctx.ys, ctx.marks = xs, ys, marks
        ctx.save_for_backward(*params)
        return x.clone()

    @staticmethod
    def backward(ctx, gout):
        hd, sched, f, S = ctx.hd, ctx.schedule, ctx.f, ctx.checkpoint
        params = ctx.saved_tensors
        T = len(sched)
        pbar = [torch.zeros_like(p) for p in params]
        xbar = {T + 1: gout.detach().to(hd.torch_dtype)}

        def add(i, v):
            if v is not None:
                xbar[i] = xbar[i] + v if i in xbar else v

        def reverse(t, x_t, x_prev, y_t, pass_x):
            yl = y_t.detach().requires_grad_(True)
            xl = x_t.detach().requires_grad_(True)
            pl = None if x_prev is None else x_prev.detach().requires_grad_(True)
            ql = [p.detach().requires_grad_(p.requires_grad) for p in params]
            with torch.enable_grad():
                out = f(t, yl, xl, pl, *ql)
                ins = [yl, xl] + ([pl] if pl is not None else []) + [q for q in ql if q.requires_grad]
                gout_t = xbar.pop(t + 1)
                # an f_t whose output does not depend on its inputs (e.g. a constant) passes nothing
                g = (torch.autograd.grad(out, ins, gout_t, allow_unused=True) if out.requires_grad
                     else [None] * len(ins))
            ybar = g[0] if g[0] is not None else torch.zeros_like(yl)
            add(t, g[1])
            k = 2
            if pl is not None:
                add(t - 1, g[2])
                k = 3
            it = iter(g[k:])
            for i, p in enumerate(params):
                if p.requires_grad:
                    gp = next(it)
                    if gp is not None:
                        pbar[i] += gp
            xh = hd.adjoint_step(ybar.contiguous(), bool(sched[t - 1]),
                                 x_t.contiguous() if pass_x else None)
            add(t, xh)

        if S is None:
            for t in range(T, 0, -1):
                reverse(t, ctx.xs[t - 1], ctx.xs[t - 2] if t >= 2 else None, ctx.ys[t - 1], False)
        else:
            starts = sorted(ctx.marks)
            for a in reversed(starts):
                b = min(T, a + S - 1)
                x, xprev = ctx.marks[a]
                seg = []
                with torch.no_grad():
                    for t in range(a, b + 1):
                        y, _ = hd.probe(x, bool(sched[t - 1]), step=t)
                        seg.append((x, xprev, y))
                        x, xprev = f(t, y, x, xprev, *params), x
                for t in range(b, a - 1, -1):
                    x_t, x_prev, y_t = seg[t - a]
                    reverse(t, x_t, x_prev, y_t, True)
        x1bar = xbar.pop(1)
        grads = [None, None, None, None, x1bar]
        grads += [pbar[i] if p.requires_grad else None for i, p in enumerate(params)]
        return tuple(grads)


def trajectory(hd, x1, schedule, f, params=(), checkpoint=None):
    """x_{T+1} of the dynamics on `hd` (see the module docstring), differentiable in x1 and params.

    schedule: sequence of T booleans (True: the step uses Q^T).  f(t, y, x, x_prev, *params)
    returns x_{t+1} from torch ops; x_prev is None at t = 1.  checkpoint: None (record every
    step) or a segment length S (recompute segments in backward).
    """
    if checkpoint is not None and checkpoint < 1:
        raise ValueError("checkpoint must be a positive segment length")
    return _Trajectory.apply(hd, tuple(bool(s) for s in schedule), f, checkpoint, x1, *params)
