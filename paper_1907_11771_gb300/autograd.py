"""PyTorch autograd over the GBS library's discrete adjoint (argument marshalling only).

* ``GBSStepFn``: y_out = M(kappa)^n y_in for n macro-steps; its backward calls
  ``gbs_adjoint_step`` once per macro-step (recomputing the intermediate states
  from y_in: all n of them, or with ``snapshots=s`` at most s held at once on a
  binomial schedule), returning d/dy_in and d/dkappa.
* ``gbs_misfit_and_grad``: the receiver misfit
      J = 1/2 sum_m sum_r (p(x_r, t_m) - d_r(t_m))^2,  m = 1..n_macro,
  and dJ/dkappa, with two-level checkpointing: the forward sweep keeps every
  ``checkpoint_every``-th state; the backward sweep walks the segments in
  reverse, recomputes each segment's states from its checkpoint, and runs the
  adjoint macro-steps backwards through it (residuals injected at each
  macro-step end).  Memory: n_macro / C + C states instead of n_macro.
  With ``snapshots=s`` it follows a binomial ("revolve") schedule instead
  (``checkpoint.revolve_plan``): s + 1 states, and the least number of
  recomputed macro-steps that s stored states allow.
* ``GBSMisfitFn``: the same as an autograd Function of kappa.

Every computation runs in libgbs.so; tensors only carry memory.
"""
import torch

from . import binding as B
from .checkpoint import WORK, revolve_plan


def _stream():
    return torch.cuda.current_stream().cuda_stream


class GBSStepFn(torch.autograd.Function):
    """y_out = (macro-step)^n_macro (y_in) with gradients for y_in and kappa.

    ``solver`` must have been created with enable_adjoint=True and media whose
    kappa tensor is the ``kappa`` argument (the library reads it in place)."""

    @staticmethod
    def forward(ctx, y_in, kappa, solver, H, n_macro, snapshots=None):
        if kappa.data_ptr() != solver._media[0].data_ptr():
            raise ValueError("kappa must be the tensor the solver was created with")
        y_out = torch.empty_like(y_in)
        solver.step(y_in.detach(), y_out, H, n_macro)
        ctx.solver, ctx.H, ctx.n_macro, ctx.snapshots = solver, H, n_macro, snapshots
        ctx.save_for_backward(y_in.detach())
        return y_out

    @staticmethod
    def backward(ctx, lam_out):
        (y_in,) = ctx.saved_tensors
        sol, H, n = ctx.solver, ctx.H, ctx.n_macro
        lam = lam_out.detach().contiguous().clone()
        grad = torch.zeros(sol.state_elems // sol.F, dtype=torch.float64, device=y_in.device)
        if ctx.snapshots is None:
            states = [y_in]
            for _ in range(n - 1):
                nxt = torch.empty_like(y_in)
                sol.step(states[-1], nxt, H, 1)
                states.append(nxt)
            for m in range(n - 1, -1, -1):
                sol.adjoint_step(states[m], lam, lam, grad, H)
        else:
            # binomial schedule: the first descent's states stored by a forward sweep, then the
            # plan's advances and adjoint macro-steps (checkpoint.revolve_plan)
            plan = revolve_plan(n, int(ctx.snapshots))
            slots = [y_in.clone()] + [torch.empty_like(y_in) for _ in range(plan.max_slots - 1)]
            work = y_in.clone()
            buf = lambda k: work if k == WORK else slots[k]
            stores = dict(plan.forward_stores)
            for m in range(max(stores, default=0)):
                sol.step(work, work, H, 1)
                if (m + 1) in stores:
                    slots[stores[m + 1]].copy_(work)
            for act in plan.actions:
                if act[0] == "advance":
                    _, src, dst, a, m = act
                    sol.step(buf(src), buf(dst), H, m - a)
                else:
                    _, k, m = act
                    sol.adjoint_step(buf(k), lam, lam, grad, H)
        return lam, grad.to(y_in.dtype), None, None, None, None


def gbs_misfit_and_grad(solver, y0, H, n_macro, rcv_idx, data, checkpoint_every=50, snapshots=None):
    """Return (J, dJ/dkappa as an FP64 tensor) for ``n_macro`` macro-steps from y0.

    rcv_idx: int64 device tensor of flat grid indices (field 0 of a single problem);
    data: device tensor (n_macro, n_rcv) of observed pressures at macro-step ends.
    snapshots: None for two-level checkpointing every ``checkpoint_every`` macro-steps,
    else the number of stored states of a binomial schedule (y_0 included)."""
    if snapshots is not None:
        return _misfit_and_grad_revolve(solver, y0, H, n_macro, rcv_idx, data, int(snapshots))
    C = max(1, int(checkpoint_every))
    dev = y0.device
    n_rcv = rcv_idx.numel()
    J = torch.zeros(1, dtype=torch.float64, device=dev)
    resid = torch.empty(n_macro, n_rcv, dtype=y0.dtype, device=dev)
    # forward sweep: checkpoints at m = 0, C, 2C, ...
    ckpt = {0: y0.detach().clone()}
    y = y0.detach().clone()
    for m in range(n_macro):
        solver.step(y, y, H, 1)
        solver.misfit(y, rcv_idx, data[m], resid[m], J)
        if (m + 1) % C == 0 and (m + 1) < n_macro:
            ckpt[m + 1] = y.clone()
    # backward sweep over segments [s0, s1).  lam = dJ/dy_(m+1) entering macro-step m;
    # gbs_adjoint_step returns dJ/dy_m = M^T lam + (residual injected at t_m).
    grad = torch.zeros(solver.state_elems // solver.F, dtype=torch.float64, device=dev)
    lam = torch.zeros_like(y0)
    solver.inject(lam, rcv_idx, resid[n_macro - 1])          # lam_M = S^T r_M
    starts = sorted(ckpt.keys())
    for s0 in reversed(starts):
        s1 = min(s0 + C, n_macro)
        states = [ckpt[s0]]
        for _ in range(s1 - s0 - 1):
            nxt = torch.empty_like(y0)
            solver.step(states[-1], nxt, H, 1)
            states.append(nxt)
        for m in range(s1 - 1, s0 - 1, -1):
            _adjoint_macro_step(solver, states[m - s0], lam, grad, H, m, rcv_idx, resid)
        del states
    solver.sync()
    return float(J.item()), grad


def _adjoint_macro_step(solver, y_m, lam, grad, H, m, rcv_idx, resid):
    """lam <- dJ/dy_m from dJ/dy_(m+1): the adjoint of macro-step m, plus the residual at t_m."""
    if m >= 1:
        solver.adjoint_step(y_m, lam, lam, grad, H, rcv_idx, resid[m - 1])
    else:
        solver.adjoint_step(y_m, lam, lam, grad, H)


def _misfit_and_grad_revolve(solver, y0, H, n_macro, rcv_idx, data, s):
    """gbs_misfit_and_grad with s stored states placed by a binomial schedule."""
    plan = revolve_plan(n_macro, s)
    dev = y0.device
    J = torch.zeros(1, dtype=torch.float64, device=dev)
    resid = torch.empty(n_macro, rcv_idx.numel(), dtype=y0.dtype, device=dev)
    slots = [y0.detach().clone()] + [torch.empty_like(y0) for _ in range(plan.max_slots - 1)]
    work = y0.detach().clone()
    buf = lambda k: work if k == WORK else slots[k]
    stores = dict(plan.forward_stores)
    # forward sweep: misfit at every macro-step end, the first descent's states stored on the way
    for m in range(n_macro):
        solver.step(work, work, H, 1)
        solver.misfit(work, rcv_idx, data[m], resid[m], J)
        if (m + 1) in stores:
            slots[stores[m + 1]].copy_(work)
    grad = torch.zeros(solver.state_elems // solver.F, dtype=torch.float64, device=dev)
    lam = torch.zeros_like(y0)
    solver.inject(lam, rcv_idx, resid[n_macro - 1])
    for act in plan.actions:
        if act[0] == "advance":
            _, src, dst, a, m = act
            solver.step(buf(src), buf(dst), H, m - a)
        else:
            _, k, m = act
            _adjoint_macro_step(solver, buf(k), lam, grad, H, m, rcv_idx, resid)
    solver.sync()
    return float(J.item()), grad


class GBSMisfitFn(torch.autograd.Function):
    """J(kappa) = receiver misfit after n_macro macro-steps; backward gives dJ/dkappa."""

    @staticmethod
    def forward(ctx, kappa, solver, y0, H, n_macro, rcv_idx, data, checkpoint_every, snapshots=None):
        if kappa.data_ptr() != solver._media[0].data_ptr():
            raise ValueError("kappa must be the tensor the solver was created with")
        J, g = gbs_misfit_and_grad(solver, y0, H, n_macro, rcv_idx, data, checkpoint_every, snapshots)
        ctx.save_for_backward(g)
        return torch.tensor(J, dtype=torch.float64, device=kappa.device)

    @staticmethod
    def backward(ctx, gJ):
        (g,) = ctx.saved_tensors
        return (gJ * g).to(torch.float64), None, None, None, None, None, None, None, None
