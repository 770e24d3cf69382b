"""``torch.autograd.Function`` over the unrolled solve: the forward pass calls ``pimpc_solve`` (a
fixed number of plain iterations from the zero start), the backward pass ``pimpc_backward`` (the
library's reverse sweep with checkpoints). Argument marshalling only; every step runs in the
CUDA library.

Tensors use the concatenated FP64 layout of the C ABI (instances in batch order): x0, q, xmin,
xmax [sum nx]; r, umin, umax [sum nu]; ref [sum N n] (one reference per stage) or [sum n] (one per
instance); outputs u [sum N nu] and x [sum N nx]. All are CUDA tensors on the solver's device.
"""
from __future__ import annotations

import numpy as np
import torch

from . import pimpc as P


class UnrolledSolve(torch.autograd.Function):
    """(u, x) = solve(x0, ref, q, r, bounds) after ``iters`` plain iterations; differentiable in
    every tensor argument. One backward per forward, before the solver runs another solve."""

    @staticmethod
    def forward(ctx, solver, iters, checkpoint_every, x0, ref, q, r, xmin, xmax, umin, umax):
        dev = x0.device
        h = solver.h
        rdu = solver.p["rdu"]
        rdu_t = None if rdu is None else torch.from_numpy(rdu).to(dev)
        P.pimpc_set_weights(h, q.contiguous(), r.contiguous(), rdu_t)
        P.pimpc_set_bounds(h, xmin.contiguous(), xmax.contiguous(), umin.contiguous(),
                           umax.contiguous())
        P.pimpc_set_options(h, solver.p["rho"], -1.0, int(iters), 0)
        tot_u = int(np.sum(solver.N * solver.nu))
        tot_x = int(np.sum(solver.N * solver.nx))
        tot_Nn = int(np.sum(solver.N * (solver.nx + solver.nu)))
        per_stage = ref.numel() == tot_Nn and tot_Nn != int(np.sum(solver.nx + solver.nu))
        u = torch.empty(tot_u, dtype=torch.float64, device=dev)
        x = torch.empty(tot_x, dtype=torch.float64, device=dev)
        up = solver.p["u_prev"]
        up_t = None if up is None else torch.from_numpy(up).to(dev)
        P.pimpc_solve(h, x0.contiguous(), up_t, ref.contiguous(), per_stage, 0, u, x)
        solver._solve_token = getattr(solver, "_solve_token", 0) + 1
        ctx.solver = solver
        ctx.token = solver._solve_token
        ctx.K = int(checkpoint_every)
        ctx.shapes = (x0.shape, ref.shape, q.shape, r.shape, xmin.shape, xmax.shape, umin.shape,
                      umax.shape)
        return u, x

    @staticmethod
    def backward(ctx, gu, gx):
        solver = ctx.solver
        if getattr(solver, "_solve_token", None) != ctx.token:
            raise RuntimeError("the solver ran another solve after this forward pass")
        need = ctx.needs_input_grad[3:]
        dev = gu.device if gu is not None else gx.device
        outs = [torch.zeros(s, dtype=torch.float64, device=dev) if nd else None
                for s, nd in zip(ctx.shapes, need)]
        g_x0, g_ref, g_q, g_r, g_xmin, g_xmax, g_umin, g_umax = outs
        P.pimpc_backward(solver.h, None if gu is None else gu.contiguous(),
                         None if gx is None else gx.contiguous(), g_x0, g_ref, g_q, g_r, g_xmin,
                         g_xmax, g_umin, g_umax, ctx.K)
        return (None, None, None) + tuple(outs)


def unrolled_solve(solver, iters, x0, ref, q, r, xmin, xmax, umin, umax, checkpoint_every=25):
    """Functional form of ``UnrolledSolve.apply``."""
    return UnrolledSolve.apply(solver, iters, checkpoint_every, x0, ref, q, r, xmin, xmax, umin,
                               umax)
