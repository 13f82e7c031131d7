"""torch.autograd.Function for x*(b, c) of a batch of LPs  min c^T x, Ax = b, x >= 0.

Forward: batched restarted PDHG to eps_rel, then the active-set polish
(pdhg_batch_polish).  Backward: the vector-Jacobian product of the
active-set fixed point (pdhg_batch_adjoint): dL/db = A_B (A_B^T A_B)^{-1}
dL/dx_B, dL/dc = 0.  Both run in the library's CUDA kernels; nothing is
unrolled, so no checkpointing is needed.
"""
from __future__ import annotations

import numpy as np
import torch

from . import pdhg


class LPSolution(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, c, structure, eps_rel=1e-4, max_iter=200_000, cg_tol=1e-12,
                cg_max_iter=5000, precision="fp64"):
        """b: float64 [sum m], c: float64 [sum n] (CPU or CUDA tensors);
        structure: dict m, n (int32 per LP), row_ptr, col, val (concatenated,
        as pdhg_batch_create takes them; numpy arrays)."""
        dev = b.device
        arrays = dict(structure)
        arrays["b"] = b.detach().to("cpu", torch.float64).numpy()
        arrays["c"] = c.detach().to("cpu", torch.float64).numpy()
        solver = pdhg.BatchSolver(arrays=arrays, precision=precision)
        solver.solve(eps_rel, max_iter)
        pol = solver.polish(cg_tol, cg_max_iter)
        ctx.solver = solver
        ctx.cg = (cg_tol, cg_max_iter)
        ctx.device = dev
        ctx.active = pol["active"]
        return torch.from_numpy(np.array(pol["x"])).to(dev)

    @staticmethod
    def backward(ctx, grad_x):
        cg_tol, cg_max_iter = ctx.cg
        r = ctx.solver.adjoint(grad_x.detach().to("cpu", torch.float64).contiguous().numpy(),
                               cg_tol, cg_max_iter)
        gb = torch.from_numpy(np.array(r["grad_b"])).to(ctx.device)
        gc = torch.from_numpy(np.array(r["grad_c"])).to(ctx.device)
        return gb, gc, None, None, None, None, None, None


def lp_solution(b, c, structure, **kw):
    return LPSolution.apply(b, c, structure, kw.get("eps_rel", 1e-4), kw.get("max_iter", 200_000),
                            kw.get("cg_tol", 1e-12), kw.get("cg_max_iter", 5000),
                            kw.get("precision", "fp64"))
