"""Differentiable deskew: autograd Functions over the library's kernels.

* ``DeskewFn``: raw stack -> volume (the LINEAR deskew A).  Its backward is
  the skew adjoint A^T (``opm_skew_adjoint``), the exact transpose of the
  map the forward kernel applies.
* ``SkewFn``: volume -> raw stack (A^T), the forward model of an acquisition
  of a volume; its backward is A.
* ``ProjectFn``: raw stack -> z-MIP (Fig. 2d live view).  Its backward routes
  the gradient to the raw samples of the voxel that attained each maximum
  (``opm_mip_backward`` with the stored argmax).

All tensors are CUDA tensors; every forward and backward step runs in the
library's kernels.  FP64 is supported by DeskewFn/SkewFn for gradient checks.
"""
from __future__ import annotations

import torch

from . import Plan, opm_deskew, opm_mip_backward, opm_project, opm_skew_adjoint


class DeskewFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, raw: torch.Tensor, plan: Plan):
        if raw.dtype not in (torch.float32, torch.float64):
            raise TypeError("DeskewFn takes float32 or float64 stacks")
        raw = raw.contiguous()
        vol = torch.empty(plan.vol_shape, dtype=raw.dtype, device=raw.device)
        opm_deskew(plan, raw, vol)
        ctx.plan = plan
        return vol

    @staticmethod
    def backward(ctx, g):
        plan = ctx.plan
        g = g.contiguous()
        out = torch.empty(plan.raw_shape, dtype=g.dtype, device=g.device)
        opm_skew_adjoint(plan, g, out)
        return out, None


class SkewFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, vol: torch.Tensor, plan: Plan):
        vol = vol.contiguous()
        raw = torch.empty(plan.raw_shape, dtype=vol.dtype, device=vol.device)
        opm_skew_adjoint(plan, vol, raw)
        ctx.plan = plan
        return raw

    @staticmethod
    def backward(ctx, g):
        plan = ctx.plan
        g = g.contiguous()
        out = torch.empty(plan.vol_shape, dtype=g.dtype, device=g.device)
        opm_deskew(plan, g, out)
        return out, None


class ProjectFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, raw: torch.Tensor, plan: Plan):
        if raw.dtype != torch.float32:
            raise TypeError("ProjectFn takes float32 stacks")
        raw = raw.contiguous()
        zmip = torch.empty((plan.ny, plan.nx), dtype=torch.float32, device=raw.device)
        argz = torch.empty((plan.ny, plan.nx), dtype=torch.int32, device=raw.device)
        opm_project(plan, raw, zmip, None, None, argz)
        ctx.plan = plan
        ctx.save_for_backward(argz)
        ctx.mark_non_differentiable(argz)
        return zmip, argz

    @staticmethod
    def backward(ctx, g_zmip, g_argz):
        (argz,) = ctx.saved_tensors
        plan = ctx.plan
        out = torch.empty(plan.raw_shape, dtype=torch.float32, device=g_zmip.device)
        opm_mip_backward(plan, g_zmip.contiguous(), argz, out)
        return out, None


def deskew(raw, plan):
    return DeskewFn.apply(raw, plan)


def skew(vol, plan):
    return SkewFn.apply(vol, plan)


def zmip(raw, plan):
    return ProjectFn.apply(raw, plan)[0]


def power_iteration(plan: Plan, iters: int = 20, seed: int = 0, dtype=torch.float32):
    """Largest eigenvalue of A A^T (= ||A||^2) by power iteration."""
    gen = torch.Generator(device="cuda").manual_seed(seed)
    x = torch.randn(plan.raw_shape, generator=gen, device="cuda", dtype=dtype)
    x /= x.norm()
    lam = 0.0
    vol = torch.empty(plan.vol_shape, dtype=dtype, device="cuda")
    for _ in range(iters):
        opm_deskew(plan, x, vol)
        y = torch.empty_like(x)
        opm_skew_adjoint(plan, vol, y)
        lam = float(y.norm())
        x = y / lam
    return lam


def reconstruct(plan: Plan, measured: torch.Tensor, iters: int = 100, eta: float | None = None,
                x0: torch.Tensor | None = None, lipschitz: float | None = None,
                checkpoint: str | None = None, every: int = 10):
    """Gradient descent on 0.5 ||A^T x - y||^2 over volumes x (output grid).

    The gradient A (A^T x - y) is one skew (A^T) and one deskew (A) per
    iteration.  With eta <= 1/L, L = ||A||^2, the loss is non-increasing.
    Returns (x, losses).

    ``checkpoint``: a file path.  If it exists, the run resumes from the
    iterate, step size and losses stored there; every ``every`` iterations
    (and at the end) they are written there again with ``torch.save``.  A
    resumed run ends on the same iterate as an uninterrupted one: each step
    is a deterministic function of the iterate.
    """
    import os
    state = torch.load(checkpoint, map_location=measured.device) if checkpoint and os.path.exists(checkpoint) else None
    if state is not None:
        x = state["x"].to(device=measured.device, dtype=measured.dtype).clone()
        eta = float(state["eta"])
        losses = list(state["losses"])
        done = int(state["iters"])
    else:
        if lipschitz is None:
            lipschitz = power_iteration(plan)
        if eta is None:
            eta = 1.0 / lipschitz
        x = torch.zeros(plan.vol_shape, dtype=measured.dtype, device=measured.device) if x0 is None else x0.clone()
        losses = []
        done = 0
    r = torch.empty(plan.raw_shape, dtype=measured.dtype, device=measured.device)
    grad = torch.empty_like(x)

    def save(n):
        if checkpoint:
            tmp = checkpoint + ".tmp"
            torch.save({"x": x, "eta": eta, "losses": losses, "iters": n}, tmp)
            os.replace(tmp, checkpoint)

    for it in range(done, iters):
        opm_skew_adjoint(plan, x, r)
        r.sub_(measured)
        losses.append(0.5 * float(r.double().pow(2).sum()))
        opm_deskew(plan, r, grad)
        x.add_(grad, alpha=-eta)
        if checkpoint and (it + 1) % every == 0:
            save(it + 1)
    opm_skew_adjoint(plan, x, r)
    r.sub_(measured)
    final = 0.5 * float(r.double().pow(2).sum())
    save(max(done, iters))
    return x, losses + [final]
