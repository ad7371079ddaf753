"""torch.autograd binding of the flow rate as a function of the per-cell collision rate.

FlowRate.apply(delta, solver) runs the source iteration of Eq. (iteration) with delta_c as the
collision rate of every gas cell and returns Q (Sec. III, Eq. Q); backward runs the adjoint of the
projected iteration (dvm_adjoint) for dQ/d delta_c.  All arithmetic runs in libdvm; torch only carries
the tensors.  The solver must keep its distribution (store_distribution=True).
"""
from __future__ import annotations

import numpy as np
import torch

from . import dvm


class FlowRate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, delta, solver, tol=1e-12, max_iter=100000, adjoint_tol=1e-12):
        if tuple(delta.shape) != tuple(solver.shape):
            raise ValueError(f"delta field shape {tuple(delta.shape)} != grid {solver.shape}")
        solver.set_delta_field(delta.detach().to("cpu", torch.float64).numpy())
        solver.solve(tol=tol, max_iter=max_iter)
        q, _ = solver.flowrate()
        ctx.solver = solver
        ctx.adjoint = (adjoint_tol, max_iter)
        return torch.tensor(q, dtype=delta.dtype, device=delta.device)

    @staticmethod
    def backward(ctx, grad_q):
        tol, max_iter = ctx.adjoint
        g, _, _ = ctx.solver.adjoint(tol=tol, max_iter=max_iter)
        grad = torch.from_numpy(np.ascontiguousarray(g)).to(device=grad_q.device, dtype=grad_q.dtype)
        return grad_q * grad, None, None, None, None


def flow_rate(delta, solver, tol=1e-12, max_iter=100000, adjoint_tol=1e-12):
    """Q(delta) with autograd support (see FlowRate)."""
    return FlowRate.apply(delta, solver, tol, max_iter, adjoint_tol)
