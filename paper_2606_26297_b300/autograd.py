"""torch.autograd.Function for the QAOA objective E(gamma, beta).

The forward call runs the library's fused forward + adjoint sweep
(qaoa_grad) once and keeps the exact gradient; backward only scales it by the
incoming gradient.  The objective is the mean cost of Sec. 3.4
(Eq. training_objective_mean_cost), evaluated exactly on the statevector.
"""
from __future__ import annotations

import torch

from . import qaoa as _q


class QaoaExpectation(torch.autograd.Function):
    @staticmethod
    def forward(fctx, gamma: torch.Tensor, beta: torch.Tensor, ctx_handle, cost_handle):
        g = gamma.detach().to("cpu", torch.float64).numpy()
        b = beta.detach().to("cpu", torch.float64).numpy()
        E, dg, db = _q.qaoa_grad(ctx_handle, cost_handle, g, b)
        fctx.save_for_backward(torch.from_numpy(dg).to(gamma.device, gamma.dtype),
                               torch.from_numpy(db).to(beta.device, beta.dtype))
        return torch.tensor(E, dtype=gamma.dtype, device=gamma.device)

    @staticmethod
    def backward(fctx, grad_out):
        dg, db = fctx.saved_tensors
        return grad_out * dg, grad_out * db, None, None


def qaoa_expectation(gamma: torch.Tensor, beta: torch.Tensor, ctx_handle, cost_handle) -> torch.Tensor:
    return QaoaExpectation.apply(gamma, beta, ctx_handle, cost_handle)


class QaoaExpectationBatch(torch.autograd.Function):
    """E_b(gamma_b, beta_b) for B parameter sets (tensors of shape (B, p)) in
    one batched request (qaoa_grad_batch); item b uses costs[item_cost[b]]."""

    @staticmethod
    def forward(fctx, gamma: torch.Tensor, beta: torch.Tensor, ctx_handle, costs, item_cost):
        g = gamma.detach().to("cpu", torch.float64).numpy()
        b = beta.detach().to("cpu", torch.float64).numpy()
        E, dg, db = _q.qaoa_grad_batch(ctx_handle, costs, g, b, item_cost=item_cost)
        fctx.save_for_backward(torch.from_numpy(dg).to(gamma.device, gamma.dtype),
                               torch.from_numpy(db).to(beta.device, beta.dtype))
        return torch.from_numpy(E).to(gamma.device, gamma.dtype)

    @staticmethod
    def backward(fctx, grad_out):
        dg, db = fctx.saved_tensors
        w = grad_out.reshape(-1, 1)
        return w * dg, w * db, None, None, None


def qaoa_expectation_batch(gamma: torch.Tensor, beta: torch.Tensor, ctx_handle, costs,
                           item_cost=None) -> torch.Tensor:
    return QaoaExpectationBatch.apply(gamma, beta, ctx_handle, costs, item_cost)
