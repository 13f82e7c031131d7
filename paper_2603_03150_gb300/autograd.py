"""torch.autograd.Function for x*(b, c) of a batch of LPs  min c^T x, Ax = b, x >= 0.

Forward: batched restarted PDHG to eps_rel, then the active-set polish
(pdhg_batch_polish).  Backward: the vector-Jacobian product of the
active-set fixed point (pdhg_batch_adjoint): dL/db = A_B (A_B^T A_B)^{-1}
dL/dx_B, dL/dc = 0.  Both run in the library's CUDA kernels; nothing is
unrolled, so no checkpointing is needed.

``BatchLP`` holds one library context per structure (A): it uploads A once,
and its scaling, transpose, power iteration and tile schedules are reused by
every call, which only sends new b and c (pdhg_batch_set_rhs).  With CUDA
tensors b and c the whole call stays on the device: b, c, x and the
gradients are device tensors passed to the library by pointer.
"""
from __future__ import annotations

import numpy as np
import torch

from . import pdhg


class BatchLP:
    """A batch of LPs with fixed A (``structure``: dict m, n int32 per LP and
    the concatenated row_ptr, col, val as pdhg_batch_create takes them) whose
    b, c change from call to call.  ``device="cuda"`` keeps A, b, c, x and the
    gradients on the GPU."""

    def __init__(self, structure, device="cuda", precision: str = "fp64"):
        self.structure = structure
        self.device = torch.device(device)
        self.precision = precision
        self.on_device = self.device.type == "cuda"
        self.solver = None
        self._arrays = None
        self.generation = 0  # forward calls so far (a backward needs its own)

    def _host_or_device(self, a, dtype):
        t = a if torch.is_tensor(a) else torch.from_numpy(np.ascontiguousarray(a))
        t = t.to(dtype)
        return t.to(self.device).contiguous() if self.on_device else t.cpu().contiguous()

    def _prepare(self, b, c):
        """The library context (created on the first call) with this b, c."""
        if self.solver is None:
            st = self.structure
            arrays = dict(m=np.asarray(st["m"], np.int32), n=np.asarray(st["n"], np.int32),
                          row_ptr=self._host_or_device(st["row_ptr"], torch.int32),
                          col=self._host_or_device(st["col"], torch.int32),
                          val=self._host_or_device(st["val"], torch.float64), b=b, c=c)
            self._arrays = arrays
            self.solver = pdhg.BatchSolver(arrays=arrays, precision=self.precision,
                                           device_io=self.on_device)
        else:
            self.solver.set_rhs(b, c)
        self.generation += 1
        return self.solver

    def close(self):
        if self.solver is not None:
            self.solver.close()
            self.solver = None


class LPSolution(torch.autograd.Function):
    @staticmethod
    def forward(ctx, b, c, lp, eps_rel=1e-4, max_iter=200_000, cg_tol=1e-12,
                cg_max_iter=5000, precision="fp64"):
        """b: float64 [sum m], c: float64 [sum n]; lp: a BatchLP (reused
        across calls), or a structure dict (a context for this call only)."""
        dev = b.device
        own = not isinstance(lp, BatchLP)
        if own:
            lp = BatchLP(lp, device=dev, precision=precision)
        bd = lp._host_or_device(b.detach(), torch.float64)
        cd = lp._host_or_device(c.detach(), torch.float64)
        solver = lp._prepare(bd, cd)
        solver.solve(eps_rel, max_iter)
        pol = solver.polish(cg_tol, cg_max_iter)
        ctx.lp = lp
        ctx.generation = lp.generation
        ctx.own = own
        ctx.cg = (cg_tol, cg_max_iter)
        ctx.device = dev
        ctx.active = pol["active"]
        x = pol["x"]
        return x.to(dev) if torch.is_tensor(x) else torch.from_numpy(np.array(x)).to(dev)

    @staticmethod
    def backward(ctx, grad_x):
        cg_tol, cg_max_iter = ctx.cg
        lp = ctx.lp
        if lp.generation != ctx.generation:
            raise RuntimeError("this BatchLP solved another b, c after this forward; give "
                               "each solution that needs a backward its own BatchLP")
        g = lp._host_or_device(grad_x.detach(), torch.float64)
        if not lp.on_device:
            g = g.numpy()
        r = lp.solver.adjoint(g, cg_tol, cg_max_iter)
        as_t = lambda a: a.to(ctx.device) if torch.is_tensor(a) else torch.from_numpy(np.array(a)).to(ctx.device)
        gb, gc = as_t(r["grad_b"]), as_t(r["grad_c"])
        if ctx.own:
            lp.close()
        return gb, gc, None, None, None, None, None, None


def lp_solution(b, c, lp, **kw):
    return LPSolution.apply(b, c, lp, kw.get("eps_rel", 1e-4), kw.get("max_iter", 200_000),
                            kw.get("cg_tol", 1e-12), kw.get("cg_max_iter", 5000),
                            kw.get("precision", "fp64"))
