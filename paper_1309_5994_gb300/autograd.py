"""torch.autograd bridge to the adjoint: differentiable weighted site observables.

    L = sum_i w_i n_i(t_k) + v_i D_i(t_k)      (densities and double occupancies)

as a function of the drive tables U [Nr, Nt] and J [Nb, Nt] (float64 torch
tensors).  The forward pass calls the C ABI's dyson_adjoint (forward columns,
transposed-block rows and gradient contractions all run on the GPU) and keeps
the gradients; the backward pass scales them by the incoming gradient.  Any
scalar drive parameter from which U and J are built with torch operations
(for example an amplitude s in U = U0 (1 + a s sin wt)) then receives its
gradient through torch's chain rule.
"""
from __future__ import annotations

import torch

from . import binding


class WeightedObservables(torch.autograd.Function):
    @staticmethod
    def forward(ctx, U, J, problem, w, v, t_index, precision, tol):
        p = problem.with_tables(U=U.detach().cpu().numpy(), J=J.detach().cpu().numpy())
        solver = binding.Solver(p, device=torch.cuda.current_device())
        solver.build_sigma()
        loss, gU, gJ, _ = solver.adjoint_obs(w, v, t_index=t_index, precision=precision, tol=tol)
        solver.close()
        ctx.save_for_backward(torch.from_numpy(gU).to(U), torch.from_numpy(gJ).to(J))
        return torch.tensor(loss, dtype=torch.float64, device=U.device)

    @staticmethod
    def backward(ctx, grad_out):
        gU, gJ = ctx.saved_tensors
        return grad_out * gU, grad_out * gJ, None, None, None, None, None, None


def weighted_observables(U, J, problem, w=None, v=None, t_index=None, precision=binding.PREC_TF32X3_F64REF,
                         tol=1e-11):
    """Differentiable L = sum_i w_i n_i(t_index) + v_i D_i(t_index) (default: the last forward time)."""
    t_index = problem.Nt - 1 if t_index is None else t_index
    return WeightedObservables.apply(U, J, problem, w, v, t_index, precision, tol)


def weighted_density(U, J, problem, w, t_index=None, precision=binding.PREC_TF32X3_F64REF, tol=1e-11):
    """Differentiable L = sum_i w_i n_i(t_index) (default: the last forward time)."""
    return weighted_observables(U, J, problem, w=w, t_index=t_index, precision=precision, tol=tol)
