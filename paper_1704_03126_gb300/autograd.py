"""torch.autograd binding of the flow rate as a function of the per-cell collision rate.

FlowRate.apply(delta, solver) runs the source iteration of Eq. (iteration) with delta_c as the
collision rate of every gas cell and returns Q (Sec. III, Eq. Q); backward runs the adjoint of the
projected iteration (dvm_adjoint) for dQ/d delta_c.  All arithmetic runs in libdvm; torch only carries
the tensors.  The solver must keep its distribution (store_distribution=True).

One solver may serve several graph nodes: forward records the delta field it solved for and the
solver's state id, and backward re-solves at that field first when the solver has been used since
(for example forward(d1), forward(d2), backward of the first).  An adjoint iteration that runs out of
sweeps raises (allow_noconv=True turns that into a warning).
"""
from __future__ import annotations

import warnings

import numpy as np
import torch

from . import dvm


class FlowRate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, delta, solver, tol=1e-12, max_iter=100000, adjoint_tol=1e-12, allow_noconv=False,
                adjoint_max_iter=None):
        if tuple(delta.shape) != tuple(solver.shape):
            raise ValueError(f"delta field shape {tuple(delta.shape)} != grid {solver.shape}")
        field = np.ascontiguousarray(delta.detach().to("cpu", torch.float64).numpy()).copy()
        solver.set_delta_field(field)
        solver.solve(tol=tol, max_iter=max_iter)
        q, _ = solver.flowrate()
        ctx.solver = solver
        ctx.field = field
        ctx.state_id = solver.state_id
        ctx.forward_args = (tol, max_iter)
        ctx.adjoint = (adjoint_tol, max_iter if adjoint_max_iter is None else adjoint_max_iter, allow_noconv)
        return torch.tensor(q, dtype=delta.dtype, device=delta.device)

    @staticmethod
    def backward(ctx, grad_q):
        tol, max_iter, allow_noconv = ctx.adjoint
        solver = ctx.solver
        if solver.state_id != ctx.state_id:
            # the solver has moved on since this node's forward: restore the state it differentiates
            solver.set_delta_field(ctx.field)
            solver.solve(tol=ctx.forward_args[0], max_iter=ctx.forward_args[1])
            ctx.state_id = solver.state_id
        g, _, _ = solver.adjoint(tol=tol, max_iter=max_iter)
        if solver.last_adjoint_status == dvm.DVM_ENOCONV:
            msg = f"adjoint iteration did not reach tol {tol:g} in {max_iter} sweeps: dQ/d delta is inexact"
            if not allow_noconv:
                raise dvm.DvmError(dvm.DVM_ENOCONV, msg)
            warnings.warn(msg, RuntimeWarning)
        grad = torch.from_numpy(np.ascontiguousarray(g)).to(device=grad_q.device, dtype=grad_q.dtype)
        return grad_q * grad, None, None, None, None, None, None


def flow_rate(delta, solver, tol=1e-12, max_iter=100000, adjoint_tol=1e-12, allow_noconv=False,
              adjoint_max_iter=None):
    """Q(delta) with autograd support (see FlowRate); adjoint_max_iter defaults to max_iter."""
    return FlowRate.apply(delta, solver, tol, max_iter, adjoint_tol, allow_noconv, adjoint_max_iter)
