"""torch.autograd.Function around the adjoint kernel of the OT-weighted spot
cost.

E_n(w, x) = sum_{j in J_n} sum_i Q_ij C_ij(exp([w_n]x) R0_n, x_n), with the
plan Q held at the potentials of an E-step (by Danskin's theorem this is the
gradient of the converged entropic OT value).  The forward pass refreshes the
frozen model list at the perturbed poses and evaluates E with
laue_objective_grad; it keeps the poses, not the gradient.  The backward pass
calls laue_objective_grad again, recomputing every cost on the device (costs
are never stored), and maps the left-perturbation gradient to (w, x) with
laue_axis_angle_vjp.
"""
from __future__ import annotations

import torch

from . import api


class OTWeightedCost(torch.autograd.Function):
    @staticmethod
    def forward(ctx, w, x, R0, h, geom, lat, obs, model, f, g, eps, omega):
        wd = w.detach().float().contiguous()
        xd = x.detach().float().contiguous()
        R = api.axis_angle(h, wd, R0)
        api.refresh(h, geom, lat, R, xd, omega, model)
        _, val = api.objective_grad(h, geom, lat, obs, model, f, g, eps, omega, R, xd)
        ctx.save_for_backward(wd, xd, R, f, g, omega)
        ctx.rest = (h, geom, lat, obs, model, eps)
        return val.clone()

    @staticmethod
    def backward(ctx, gout):
        wd, xd, R, f, g, omega = ctx.saved_tensors
        h, geom, lat, obs, model, eps = ctx.rest
        if not any(ctx.needs_input_grad[:2]):
            return (None,) * 12
        # the model list may have been refreshed at other poses since the forward pass
        api.refresh(h, geom, lat, R, xd, omega, model)
        grad, _ = api.objective_grad(h, geom, lat, obs, model, f, g, eps, omega, R, xd)
        gw, gx = api.axis_angle_vjp(h, wd, grad, gout.contiguous().float())
        return gw, gx, None, None, None, None, None, None, None, None, None, None


def ot_weighted_cost(w, x, R0, h, geom, lat, obs, model, f, g, eps, omega):
    """E (N,) as a differentiable function of the axis-angle perturbations w
    (N, 3) and the positions x (N, 3)."""
    return OTWeightedCost.apply(w, x, R0, h, geom, lat, obs, model, f, g, eps, omega)
