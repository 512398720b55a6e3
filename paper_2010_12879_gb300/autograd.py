"""``torch.autograd`` access to the adjoint gradient of the field energy.

``field_energy(sigma, a, h, omega)`` returns J = mean over the conducting
voxels of |E|^2 (the voxel-averaged field of Eq. 1, as ``Solver.efield``
without the square root) as a 0-dim tensor that is differentiable with
respect to the voxel conductivities ``sigma`` and the edge potentials ``a``.
The forward pass builds the operator, solves Eq. 3 and runs the adjoint solve
(``spfd_energy_grad``: A lambda = G^T dJ/du with the same operator and
preconditioner), so the backward pass only scales the stored gradients.
Gradients with respect to per-tissue conductivities follow from autograd
when ``sigma`` is built from a tissue table (e.g. ``table[labels]``).

The set of conducting voxels is held fixed: the gradient of an air voxel's
conductivity is zero.
"""

from __future__ import annotations

import torch

from . import SPFD_OK, SpfdError, Solver, spfd_last_error


class _FieldEnergy(torch.autograd.Function):
    @staticmethod
    def forward(ctx, sigma, a, h, omega, tol, opts):
        sig = sigma.detach().contiguous()
        av = a.detach().contiguous()
        S = Solver(sig, h, **opts)
        try:
            psi, _, st = S.solve(av, tol)
            if st != SPFD_OK:
                raise SpfdError(st, spfd_last_error())
            J, dJda, dJds, info, st = S.energy_grad(av, psi, omega, tol)
            if st != SPFD_OK:
                raise SpfdError(st, spfd_last_error())
        finally:
            S.close()
        ctx.save_for_backward(dJds, dJda)
        ctx.adjoint_info = info
        return torch.tensor(J, dtype=torch.float64, device=sigma.device)

    @staticmethod
    def backward(ctx, gJ):
        dJds, dJda = ctx.saved_tensors
        gs = gJ * dJds if ctx.needs_input_grad[0] else None
        ga = gJ * dJda if ctx.needs_input_grad[1] else None
        return gs, ga, None, None, None, None


def field_energy(sigma: torch.Tensor, a: torch.Tensor, h: float, omega: float,
                 tol: float = 1e-10, **opts) -> torch.Tensor:
    """J = mean over conducting voxels of |E|^2, differentiable in ``sigma``
    (float64 CUDA, (nz, ny, nx)) and ``a`` (float64 CUDA, (3, nz+1, ny+1,
    nx+1)).  ``tol`` applies to both solves; ``opts`` are ``spfd_opts``
    fields (e.g. ``precision=SPFD_MIXED``)."""
    return _FieldEnergy.apply(sigma, a, float(h), float(omega), float(tol), opts)
