"""Electron density as a differentiable function of the onsite potentials.

density(V) returns n_j = (1/pi) sum_e w_e Im G^<_jj(E_e) with H = H0 + diag(V)
(2 spins and 1/(2 pi) per energy, trapezoid weights w_e), computed on the GPU
path.  Its backward pass is the adjoint of nd_density_gradient: for the
incoming weights c = dL/dn,
    dL/dV_k = (2/pi) sum_e w_e Im t_k(E_e),
where t comes from two solves with the stored factorization of each energy
chunk (recomputed in the backward pass).  torch is used for memory and the
autograd plumbing; every arithmetic step of the solves runs in the library.
"""
from __future__ import annotations

import math

import torch

from . import ndgf


class _Density(torch.autograd.Function):
    @staticmethod
    def forward(ctx, V, solver, energies, weights):
        n_e = int(energies.numel())
        chunk = solver.max_ne
        out = torch.zeros(solver.n, dtype=torch.float64, device=solver.device)
        solver.set_onsite(V.detach())
        for c0 in range(0, n_e, chunk):
            m = min(chunk, n_e - c0)
            _, Gl, _ = solver.step(energies[c0:c0 + m])
            ndgf.nd_density(Gl, weights[c0:c0 + m].contiguous(), m, solver.n, 1.0 / math.pi, 1 if c0 else 0, out)
        ctx.solver = solver
        ctx.save_for_backward(V.detach(), energies, weights)
        return out

    @staticmethod
    def backward(ctx, grad_n):
        V, energies, weights = ctx.saved_tensors
        solver = ctx.solver
        n_e = int(energies.numel())
        chunk = solver.max_ne
        grad = torch.zeros(solver.n, dtype=torch.float64, device=solver.device)
        c = grad_n.detach().to(torch.float64).contiguous()
        solver.set_onsite(V)
        for c0 in range(0, n_e, chunk):
            m = min(chunk, n_e - c0)
            solver.step(energies[c0:c0 + m])
            t = solver.density_gradient_terms(c, m)
            ndgf.nd_density(t, weights[c0:c0 + m].contiguous(), m, solver.n, 2.0 / math.pi, 1 if c0 else 0, grad)
        return grad, None, None, None


def density(V: torch.Tensor, solver, energies: torch.Tensor, weights: torch.Tensor) -> torch.Tensor:
    """n_j(V) on the GPU path, differentiable in V (solver created with adjoint=True)."""
    return _Density.apply(V, solver, energies, weights)
