"""The smoothed RSS of seeds as a differentiable PyTorch function.

comet_scan_jacobian computes, in one pass of the library's kernels, every seed's smoothed RSS
(term = w e^2 + (1 - w) lambda^2, w = sigmoid((lambda - e) / tau), e the wire's smallest residual
|D - r|, Eq. 1 with the cap smoothed) together with its gradient: dD/dtheta by forward-mode
derivatives through the recorded states and the refinement steps (envelope theorem at the point of
closest approach).  The two Functions below hand that gradient to autograd: forward calls the
kernel and keeps the gradient, backward scales it by the incoming gradient.

* ``SmoothedRSS``          -- seeds as theta = (z0, phi, p_z, p_T) [S, 4] at a common vertex (vx, vy).
* ``SmoothedRSSCartesian`` -- seeds as (x, y, z, p_x, p_y, p_z) [S, 6]; every seed starts at the
  same (x, y) (the vertex of a seed lattice); the gradient covers all six components.

FP64 and a uniform axial field only (the kernel's domain).  Nothing here computes the method: the
conversions between the seed forms and the chain-rule scaling are the only tensor operations.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import binding as B
from .scan import DeviceEvent


@dataclass
class SmoothedRSSSpec:
    """What the smoothed RSS of a turn partition depends on besides the seeds."""
    ctx: B.Context
    field: B.DeviceField
    params: B.ScanParams       # n_steps, stride, lam (the cap), tol, max_iter
    event: DeviceEvent         # float64 wires, hits, mask
    charge: int
    tau: float                 # smoothing width of the cap (m)


def _evaluate(spec: SmoothedRSSSpec, theta: torch.Tensor, vx: float, vy: float):
    f64 = dict(dtype=torch.float64, device=theta.device)
    S, W = theta.shape[0], spec.event.W
    work = torch.empty(max(S * W, 1) * B.JAC_WORK_PER_PAIR, **f64)
    srss = torch.empty(S, **f64)
    grad = torch.empty((S, 4), **f64)
    jtj = torch.empty((S, 16), **f64)
    jtr = torch.empty((S, 4), **f64)
    grad6 = torch.empty((S, 6), **f64)
    ev = spec.event
    B.comet_scan_jacobian(spec.ctx, spec.field, spec.params, theta.detach().contiguous(), vx, vy,
                          spec.charge, ev.wires, ev.hit_offsets, ev.drift, ev.mask, spec.tau, work,
                          srss, grad, jtj, jtr, n_wires=W, grad6=grad6)
    return srss, grad, grad6


class SmoothedRSS(torch.autograd.Function):
    """srss[S] = SmoothedRSS.apply(theta [S, 4] float64 on the GPU, spec, vx, vy)."""

    @staticmethod
    def forward(fctx, theta, spec: SmoothedRSSSpec, vx: float, vy: float):
        if theta.dtype != torch.float64 or theta.dim() != 2 or theta.shape[1] != 4:
            raise ValueError("theta must be a float64 [S, 4] tensor")
        srss, grad, _ = _evaluate(spec, theta, vx, vy)
        fctx.save_for_backward(grad)
        return srss

    @staticmethod
    def backward(fctx, g):
        (grad,) = fctx.saved_tensors
        return g[:, None] * grad, None, None, None


class SmoothedRSSCartesian(torch.autograd.Function):
    """srss[S] = SmoothedRSSCartesian.apply(seeds [S, 6] float64 on the GPU, spec)."""

    @staticmethod
    def forward(fctx, seeds, spec: SmoothedRSSSpec):
        if seeds.dtype != torch.float64 or seeds.dim() != 2 or seeds.shape[1] != 6:
            raise ValueError("seeds must be a float64 [S, 6] tensor")
        xy = seeds[:, :2].detach()
        vx, vy = float(xy[0, 0]), float(xy[0, 1])
        if not bool(((xy[:, 0] == vx) & (xy[:, 1] == vy)).all()):
            raise ValueError("every seed must start at the same (x, y)")
        px, py = seeds[:, 3].detach(), seeds[:, 4].detach()
        theta = torch.stack([seeds[:, 2].detach(), torch.atan2(py, px), seeds[:, 5].detach(),
                             torch.hypot(px, py)], dim=1)
        srss, _, grad6 = _evaluate(spec, theta, vx, vy)
        fctx.save_for_backward(grad6)
        return srss

    @staticmethod
    def backward(fctx, g):
        (grad6,) = fctx.saved_tensors
        return g[:, None] * grad6, None
