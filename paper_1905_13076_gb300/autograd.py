"""The period-averaged eddy-current loss of a cable as a differentiable
function of one region's conductivity and Brauer constants.

``eddy_loss(theta, problem, region, **cfg)`` with ``theta`` a float64 tensor
(sigma, k1, k2, k3) returns the loss P [W/m] of the periodic solution as a
0-d tensor; its backward pass returns dP/dtheta from the periodic adjoint
(``pppc_adjoint``).  The forward call solves the periodic problem (PP-PC to
``tol``) and the adjoint right away, so the gradient is ready when backward
runs; only the coarse-point states are kept between the two (the fine
trajectories are recomputed inside the library).
"""

from __future__ import annotations

import copy

import numpy as np
import torch

from .solver import from_problem


def _with_theta(problem, region, theta):
    p = copy.deepcopy(problem)
    p.sigma = np.array(p.sigma, dtype=np.float64)
    p.brauer = np.array(p.brauer, dtype=np.float64)
    p.sigma[region] = float(theta[0])
    p.brauer[region] = [float(v) for v in theta[1:4]]
    return p


class EddyLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, problem, region, tol, adjoint_tol, cfg):
        th = theta.detach().cpu().double().numpy()
        with from_problem(_with_theta(problem, region, th), **cfg) as s:
            s.solve_periodic(tol=tol, kmax=200)
            loss, grad, _ = s.adjoint(region, tol=adjoint_tol)
        ctx.save_for_backward(torch.as_tensor(grad, dtype=theta.dtype, device=theta.device))
        return torch.tensor(loss, dtype=theta.dtype, device=theta.device)

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None, None, None, None, None


def eddy_loss(theta: torch.Tensor, problem, region: int, tol: float = 1e-11, adjoint_tol: float = 1e-10, **cfg):
    return EddyLoss.apply(theta, problem, region, tol, adjoint_tol, cfg)
