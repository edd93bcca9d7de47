"""``torch.autograd.Function`` around ``lb_adjoint``.

theta (float64, 20) = (u_in, sigma, nu_r, nu_b, a_1, b_1, ..., a_8, b_8): the inlet velocity,
the interfacial tension, the two viscosities and the azimuthal Fourier coefficients of the
inlet profile u_z = u_in [1 + sum_m (a_m cos m theta + b_m sin m theta)].  The forward pass
restores the lattice to a saved state, sets theta, and runs ``lb_adjoint`` (T steps forward
with checkpoints, then the reverse sweep); the gradient it returns is kept for ``backward``.
All arithmetic runs in the library's kernels; this module only moves 20 numbers.
"""
from __future__ import annotations

import torch

from . import GRAD_NAMES

SCALARS = ("u_in", "sigma", "nu_r", "nu_b")


def theta_of(params: dict) -> torch.Tensor:
    """theta from an lb_params dict (missing profile coefficients are 0)."""
    four = (list(params.get("fourier", ())) + [0.0] * 16)[:16]
    return torch.tensor([float(params.get(k, 0.0)) for k in SCALARS] + [float(v) for v in four], dtype=torch.float64)


def params_of(theta: torch.Tensor) -> dict:
    """lb_params fields set by theta."""
    t = [float(v) for v in theta.detach().cpu().reshape(-1)]
    if len(t) != len(GRAD_NAMES):
        raise ValueError(f"theta must hold {len(GRAD_NAMES)} values {GRAD_NAMES}")
    out = dict(zip(SCALARS, t[:4]))
    out["fourier"] = tuple(t[4:])
    return out


class LatticeObjective(torch.autograd.Function):
    """J(theta) = objective of the lattice state T steps after `state`."""

    @staticmethod
    def forward(ctx, theta, lattice, state, T, objective, args, checkpoint):
        lattice.load(state)
        lattice.set_params(**params_of(theta))
        J, g = lattice.adjoint(T, objective, args, checkpoint)
        ctx.save_for_backward(torch.as_tensor(g, dtype=theta.dtype, device=theta.device))
        return torch.tensor(J, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, grad_J):
        (g,) = ctx.saved_tensors
        return grad_J * g, None, None, None, None, None, None


def objective(lattice, theta: torch.Tensor, T: int, state: bytes | None = None, kind: str = "area",
              args=(1e-3,), checkpoint: int = 0) -> torch.Tensor:
    """Differentiable objective; `state` (from ``Lattice.save``) defaults to the current one."""
    if state is None:
        state = lattice.save()
    return LatticeObjective.apply(theta, lattice, state, int(T), kind, tuple(args), int(checkpoint))
