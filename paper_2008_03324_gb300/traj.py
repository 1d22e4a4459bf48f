"""Differentiable trajectory batch on the field: cubic B-spline positions with per-sample yaw,
cameras looking horizontally, objective sum of -log det I over the samples (Sec. VII-B uses
the information metrics of sampled poses as the perception cost of trajectory optimisation).

The trajectory parameterisation (a linear B-spline map and the yaw-to-quaternion map) is the
planner's side and runs in PyTorch; the FIM, its log-determinant and their derivatives with
respect to the sampled positions and an so(3) perturbation of every sample come from the
library (FifQuery -> fif_query / fif_query_backward).
"""
from __future__ import annotations

import math

import torch

from . import fif

# R_wc of a camera looking along +x with image y = -world z: columns (0,-1,0), (0,0,-1), (1,0,0)
_Q0 = (0.5, -0.5, 0.5, -0.5)   # (w, x, y, z)


def horizontal_quats(yaw: torch.Tensor) -> torch.Tensor:
    """Unit quaternions (w, x, y, z) of cameras looking horizontally along `yaw` (rotation about
    world z applied to the reference camera)."""
    h = 0.5 * yaw
    c, s = torch.cos(h), torch.sin(h)
    w0, x0, y0, z0 = _Q0
    # (c, 0, 0, s) (x) (w0, x0, y0, z0)
    return torch.stack([c * w0 - s * z0, c * x0 - s * y0, c * y0 + s * x0, c * z0 + s * w0], dim=-1)


def neg_logdet_objective(ctrl: torch.Tensor, yaw_ctrl: torch.Tensor, basis: torch.Tensor, field: fif.Field,
                         flags: int = fif.Q_METRICS):
    """ctrl [T, C, 3], yaw_ctrl [T, C], basis [S, C] -> (loss, phi, met, sign).

    loss = sum over samples with det > 0 of -log det I (camera frame).  `phi` [T*S, 3] is the
    zero so(3) perturbation of every sample; after loss.backward() it holds d loss / d phi."""
    T, C, _ = ctrl.shape
    t = torch.einsum("sc,tcd->tsd", basis, ctrl).reshape(-1, 3)
    yaw = (yaw_ctrl @ basis.T).reshape(-1)
    quat = horizontal_quats(yaw)
    phi = torch.zeros(t.shape[0], 3, device=t.device, dtype=t.dtype, requires_grad=True)
    met, sg, st = fif.FifQuery.apply(t.contiguous(), phi, quat.contiguous(), field, flags)
    mask = (sg > 0).to(met.dtype)
    loss = -(met[:, 1].nan_to_num() * mask).sum()
    return loss, phi, met, sg


def potential_cost_objective(ctrl: torch.Tensor, yaw_ctrl: torch.Tensor, basis: torch.Tensor, field: fif.Field,
                             eps: float, k_q: float, column: int = 1, flags: int = fif.Q_METRICS):
    """The information potential cost (Sec. VI-B, Eq. info_pot_cost) summed over the samples:
    loss = sum_s c(v_s), v_s = metric `column` (0 trace, 1 log|det|, 2 lambda_min) of sample s,
    with the threshold eps from fif.info_threshold.  The cost and its derivative come from the
    library's kernel, the metric gradient from the query adjoint.  Returns (loss, phi, met)."""
    T, C, _ = ctrl.shape
    t = torch.einsum("sc,tcd->tsd", basis, ctrl).reshape(-1, 3)
    yaw = (yaw_ctrl @ basis.T).reshape(-1)
    quat = horizontal_quats(yaw)
    phi = torch.zeros(t.shape[0], 3, device=t.device, dtype=t.dtype, requires_grad=True)
    met, sg, st = fif.FifQuery.apply(t.contiguous(), phi, quat.contiguous(), field, flags)
    cost = fif.InfoCost.apply(met, column, eps, k_q)
    return cost.sum(), phi, met


class GraphedObjective:
    """neg_logdet_objective and its backward pass captured once in a CUDA graph, for the many
    evaluations of one trajectory batch that an optimiser makes: the batch shape, the field and
    the flags are fixed at capture; each step() copies new control points (and yaws) into the
    captured inputs and replays the graph, which issues the same kernels (the B-spline map, the
    library's query and adjoint, the reductions) without the per-kernel launch cost of the host.
    After step(), `loss`, `ctrl_grad` and `phi_grad` hold the results (static tensors, overwritten
    by the next step)."""

    def __init__(self, ctrl: torch.Tensor, yaw_ctrl: torch.Tensor, basis: torch.Tensor, field: fif.Field,
                 flags: int = fif.Q_METRICS, warmup: int = 3):
        self.ctrl = ctrl.detach().clone().requires_grad_(True)
        self.yaw = yaw_ctrl.detach().clone()
        self.basis = basis.detach().clone()
        self.field = field
        side = torch.cuda.Stream(device=self.ctrl.device)
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):          # warm-up off the capture (allocator, lazy init)
            for _ in range(warmup):
                self.ctrl.grad = None
                loss, _, _, _ = neg_logdet_objective(self.ctrl, self.yaw, self.basis, field, flags)
                loss.backward()
        torch.cuda.current_stream().wait_stream(side)
        self.ctrl.grad = None
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.loss, self.phi, self.met, self.sign = neg_logdet_objective(self.ctrl, self.yaw, self.basis,
                                                                           field, flags)
            self.loss.backward()
        self.ctrl_grad = self.ctrl.grad
        self.phi_grad = self.phi.grad

    def step(self, ctrl: torch.Tensor = None, yaw_ctrl: torch.Tensor = None):
        """Replay with new inputs (None keeps the previous ones); returns (loss, d loss / d ctrl)."""
        with torch.no_grad():
            if ctrl is not None:
                self.ctrl.copy_(ctrl)
            if yaw_ctrl is not None:
                self.yaw.copy_(yaw_ctrl)
        self.graph.replay()
        return self.loss, self.ctrl_grad
