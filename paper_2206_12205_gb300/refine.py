"""Differentiable Fourier-interpolated power and sub-bin candidate refinement (libfdas K5).

``InterpolatedPower`` is a ``torch.autograd.Function`` over fdas_interp_power: its forward
returns P(r, z) at fractional points, and its backward applies the gradient (dP/dr, dP/dz) that
the same kernel launch computed with the adjoint sums.  The spectrum itself is not
differentiated.  ``refine`` runs fdas_refine (gradient ascent, FP32 steps and a final FP64 step).
All arithmetic runs in libfdas' kernels; torch supplies the buffers and the autograd graph.
"""
from __future__ import annotations

import torch

from . import fdas as _f


def _points(r: torch.Tensor, z: torch.Tensor) -> torch.Tensor:
    if r.shape != z.shape:
        raise ValueError(f"r and z must have the same shape, got {tuple(r.shape)} and {tuple(z.shape)}")
    return torch.stack([r.detach().reshape(-1).to(torch.float64), z.detach().reshape(-1).to(torch.float64)],
                       dim=1).contiguous()


class InterpolatedPower(torch.autograd.Function):
    """P(r, z) = |sum_k Xhat_k conj(I(k - r, z))|^2 at fractional (r, z); differentiable in r and z."""

    @staticmethod
    def forward(ctx, r, z, plan, xhat, fp64=False, k0=None):
        pts = _points(r, z)
        out = torch.empty(pts.shape[0], 3, dtype=torch.float64, device=pts.device)
        _f.fdas_interp_power(plan, xhat, pts, out, k0=k0, fp64=fp64)
        ctx.save_for_backward(out[:, 1].clone(), out[:, 2].clone())
        ctx.shape = r.shape
        ctx.dtypes = (r.dtype, z.dtype)
        return out[:, 0].reshape(r.shape).to(r.dtype)

    @staticmethod
    def backward(ctx, grad_p):
        dpdr, dpdz = ctx.saved_tensors
        g = grad_p.reshape(-1).to(torch.float64)
        gr = (g * dpdr).reshape(ctx.shape).to(ctx.dtypes[0])
        gz = (g * dpdz).reshape(ctx.shape).to(ctx.dtypes[1])
        return gr, gz, None, None, None, None


def interp_power(plan, xhat, r: torch.Tensor, z: torch.Tensor, fp64: bool = False, k0=None) -> torch.Tensor:
    """Differentiable interpolated power at (r, z) (same shape in, same shape out)."""
    return InterpolatedPower.apply(r, z, plan, xhat, fp64, k0)


def refine(plan, xhat, seeds: torch.Tensor, steps: int = 20):
    """Refine (n, 2) float64 seeds (r, z) on the device.

    Returns (points (n, 2), power (n, 3): FP64 P, dP/dr, dP/dz at each point, evals (n,))."""
    n = int(seeds.shape[0])
    dev = seeds.device
    out = torch.empty(n, 2, dtype=torch.float64, device=dev)
    power = torch.empty(n, 3, dtype=torch.float64, device=dev)
    evals = torch.empty(n, dtype=torch.int32, device=dev)
    _f.fdas_refine(plan, xhat, seeds.contiguous(), steps, out, power, evals)
    return out, power, evals
