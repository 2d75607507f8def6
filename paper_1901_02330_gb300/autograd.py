"""torch.autograd binding: (u, p) = solve(log K) with a hand-written backward.

The forward calls vem_set_log_coefficient_device + vem_solve; the backward calls
vem_adjoint, which solves the adjoint saddle-point system and contracts it
with dM/dlog K per cell on the GPU.  Argument marshalling only.
"""

from __future__ import annotations

import torch

from . import vemsolve as vs


class VemSolve(torch.autograd.Function):
    """u, p = VemSolve.apply(logK, solver) for a vemsolve.Solver created with
    device_io=1; logK is a CUDA float64 tensor with one entry per cell."""

    @staticmethod
    def forward(ctx, logK, solver):
        if not solver.options.device_io:
            raise ValueError("the solver must be created with device_io=1")
        if logK.dtype != torch.float64 or not logK.is_cuda:
            raise TypeError("logK must be a CUDA float64 tensor")
        solver.set_log_coefficient(logK.detach().contiguous())
        n_u, n_p = solver.sizes()
        u = torch.empty(n_u, dtype=torch.float64, device=logK.device)
        p = torch.empty(n_p, dtype=torch.float64, device=logK.device)
        solver.solve(u_out=u, p_out=p)
        ctx.solver = solver
        ctx.generation = solver.generation
        ctx.n_cells = logK.shape[0]
        return u, p

    @staticmethod
    def backward(ctx, gu, gp):
        solver = ctx.solver
        if solver.generation != ctx.generation:
            raise RuntimeError("the solver was used for another solve between forward and backward")
        dev = gu.device if gu is not None else gp.device
        g = torch.empty(ctx.n_cells, dtype=torch.float64, device=dev)
        solver.adjoint(None if gu is None else gu.contiguous(), None if gp is None else gp.contiguous(), out=g)
        return g, None


def solve(logK, solver):
    return VemSolve.apply(logK, solver)
