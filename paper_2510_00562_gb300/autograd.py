"""Algorithm 1 unrolled for a fixed number of passes as a differentiable
PyTorch operation: the forward pass and its gradient both run in libgsstv
(gsstv_solve, gsstv_unrolled_vjp).

    u = unrolled_geosstv(v, eps, alpha, beta, omega, iters=200)
    loss = ((u - u_ref) ** 2).mean()
    loss.backward()          # gradients for v and any tensor-valued parameter

The parameters may be Python floats (constants) or 0-dim tensors (their
gradients are returned).  The derivative is the one that holds almost
everywhere (the box, shrinkage and ball projections are piecewise smooth).
"""
from __future__ import annotations

import torch

from .solver import GRAD_PARAMS, GeoSSTVSolver


def _value(x) -> float:
    return float(x.detach().item()) if isinstance(x, torch.Tensor) else float(x)


class _Unrolled(torch.autograd.Function):
    @staticmethod
    def forward(ctx, v, eps, alpha, beta, omega, solver, iters, ckpt_every):
        prm = {k: _value(x) for k, x in zip(GRAD_PARAMS, (eps, alpha, beta, omega))}
        solver.set_params(max_iter=int(iters), tol=0.0, **prm)
        u, _, _, _ = solver.solve(v)
        ctx.solver, ctx.iters, ctx.ckpt, ctx.prm = solver, int(iters), int(ckpt_every), prm
        ctx.pdtype = [x.dtype if isinstance(x, torch.Tensor) else None for x in (eps, alpha, beta, omega)]
        ctx.save_for_backward(v)
        return u

    @staticmethod
    def backward(ctx, gu):
        (v,) = ctx.saved_tensors
        sol = ctx.solver
        sol.set_params(max_iter=ctx.iters, tol=0.0, **ctx.prm)
        sol.load(v)
        vbar, pbar = sol.unrolled_vjp(ctx.iters, gu.contiguous().float(), ctx.ckpt)
        grads = [vbar if ctx.needs_input_grad[0] else None]
        for k, i in zip(GRAD_PARAMS, range(1, 5)):
            grads.append(torch.tensor(pbar[k], dtype=ctx.pdtype[i - 1], device=v.device)
                         if ctx.needs_input_grad[i] else None)
        return tuple(grads) + (None, None, None)


def unrolled_geosstv(v: torch.Tensor, eps, alpha, beta, omega, iters: int,
                     solver: GeoSSTVSolver | None = None, ckpt_every: int = 0, **params) -> torch.Tensor:
    """u after `iters` passes of Algorithm 1 from the standard start, with
    gradients.  v: contiguous float32 CUDA tensor (N3, N1, N2).  solver: an
    FP32-storage GeoSSTVSolver of v's shape to reuse (one is made otherwise,
    with **params for the remaining fields)."""
    if solver is None:
        n3, n1, n2 = v.shape
        solver = GeoSSTVSolver(n1, n2, n3, storage="fp32", graph_iters=16, **params)
    u = _Unrolled.apply(v, eps, alpha, beta, omega, solver, iters, ckpt_every)
    return u
