"""torch.autograd.Function around the adjoint kernel of the OT-weighted spot
cost.

E_n(w, x) = sum_{j in J_n} sum_i Q_ij C_ij(exp([w_n]x) R0_n, x_n), with the
plan Q held at the potentials of an E-step (by Danskin's theorem this is the
gradient of the converged entropic OT value).  The forward pass refreshes the
frozen model list at the perturbed poses and evaluates E with
laue_objective_grad; the backward pass reuses the gradient that call computed
(costs are recomputed on the device, never stored) and maps the
left-perturbation gradient to w with the SO(3) left Jacobian.
"""
from __future__ import annotations

import torch

from . import api


class OTWeightedCost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, x, R0, h, geom, lat, obs, model, f, g, eps, omega):
        R, JlT = api.axis_angle(h, w.detach().float().contiguous(), R0, with_jacobian=True)
        xd = x.detach().float().contiguous()
        api.refresh(h, geom, lat, R, xd, omega, model)
        grad, val = api.objective_grad(h, geom, lat, obs, model, f, g, eps, omega, R, xd)
        ctx.save_for_backward(grad, JlT)
        return val.clone()

    @staticmethod
    def backward(ctx, gout):
        grad, JlT = ctx.saved_tensors
        gw = (JlT.view(-1, 3, 3) * grad[:, None, :3]).sum(-1) * gout[:, None]
        gx = grad[:, 3:] * gout[:, None]
        return gw, gx, None, None, None, None, None, None, None, None, None, None


def ot_weighted_cost(w, x, R0, h, geom, lat, obs, model, f, g, eps, omega):
    """E (N,) as a differentiable function of the axis-angle perturbations w
    (N, 3) and the positions x (N, 3)."""
    return OTWeightedCost.apply(w, x, R0, h, geom, lat, obs, model, f, g, eps, omega)
