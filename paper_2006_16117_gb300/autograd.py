"""torch.autograd.Function wrappers of the library's gradient calls.

The values of A's stored entries (a complex128 CUDA tensor, in the CSR order
the handle was created with) are the differentiable input; each forward pass
loads them into the handle (sim_update_values) and every step runs in the
library's kernels: node solves, the quadrature, the adjoint solves with
(A - zB)^H and the gradient on the stored entries.  PyTorch's convention for
a real loss L of complex inputs is ∂L/∂Re + i ∂L/∂Im, which is what the
library returns for Φ; for the holomorphic eigenvalue the backward pass
applies grad_λ · conj(dλ/da).
"""
from __future__ import annotations

import torch

from ._binding import Sim


class ProjectionNorm(torch.autograd.Function):
    """Φ(a) = ||P f||², P f = Σ_j w_j (A - z_j B)^{-1} f on the circle
    (center, radius) with `nodes` trapezoid nodes (the projection of the
    paper's Eq. XLXf).  keep=False recomputes the node solutions in the
    backward pass instead of keeping them on the device."""

    @staticmethod
    def forward(ctx, a_values, sim: Sim, center, radius, f, nodes=16, keep=True):
        sim.update_values(a_values.detach())
        phi = sim.projection_norm(center, radius, f, nodes, keep)
        ctx.sim = sim
        ctx.nnz = a_values.numel()
        return torch.tensor(phi, dtype=torch.float64, device=a_values.device)

    @staticmethod
    def backward(ctx, grad_phi):
        gA, _ = ctx.sim.projection_norm_grad(ctx.nnz, device=True)
        return grad_phi * gA, None, None, None, None, None, None


class Eigenvalue(torch.autograd.Function):
    """λ(a): the simple eigenvalue inside the circle (center, radius), as a
    complex scalar tensor, differentiable with respect to A's stored values."""

    @staticmethod
    def forward(ctx, a_values, sim: Sim, center, radius, nodes=16, seed=0x5EED):
        sim.update_values(a_values.detach())
        lam, dA, _ = sim.eigenvalue_grad(center, radius, a_values.numel(), nodes=nodes, seed=seed, device=True)
        ctx.save_for_backward(dA)
        return torch.tensor(lam, dtype=torch.complex128, device=a_values.device)

    @staticmethod
    def backward(ctx, grad_lam):
        (dA,) = ctx.saved_tensors
        return grad_lam * torch.conj(dA), None, None, None, None, None


def projection_norm(a_values, sim: Sim, center, radius, f, nodes=16, keep=True):
    return ProjectionNorm.apply(a_values, sim, center, radius, f, nodes, keep)


def eigenvalue(a_values, sim: Sim, center, radius, nodes=16, seed=0x5EED):
    return Eigenvalue.apply(a_values, sim, center, radius, nodes, seed)
