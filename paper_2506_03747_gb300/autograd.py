"""torch.autograd.Function around the differentiable splat forward and its
hand-written adjoint (both CUDA kernels behind the C ABI).

``NlosSplat.apply(albedo, depth, points, params)`` returns tau [S, B] of the
scene whose point p has albedo ``albedo[p]`` and is displaced by ``depth[p]``
metres along its normal; gradients flow to ``albedo`` and ``depth``. The
adjoint is evaluated at the displaced points, so it is exact at any depth.
"""
from __future__ import annotations

import torch

from . import nlos


def _scene(points: torch.Tensor, albedo: torch.Tensor, depth: torch.Tensor, prm):
    # displaced copy of the point records (device-side tensor arithmetic is
    # marshalling of the inputs; the simulator itself runs in libnlos.so)
    pts = points.detach().clone()
    d = depth.detach().to(pts.dtype)
    pts[:, 0:3] += d[:, None] * pts[:, 3:6]
    pts[:, 6] = albedo.detach().to(pts.dtype)
    return nlos.scene_create(prm, pts.contiguous())


class NlosSplat(torch.autograd.Function):
    @staticmethod
    def forward(ctx, albedo, depth, points, prm):
        sc = _scene(points, albedo, depth, prm)
        tau = torch.empty((sc.num_scan, sc.num_bins), dtype=torch.float32, device=points.device)
        nlos.simulate(sc, tau)
        ctx.scene = sc
        return tau

    @staticmethod
    def backward(ctx, grad_tau):
        sc = ctx.scene
        g = grad_tau.contiguous().to(torch.float32)
        ga = torch.empty(sc.num_points, dtype=torch.float32, device=g.device)
        gd = torch.empty(sc.num_points, dtype=torch.float32, device=g.device)
        nlos.simulate_backward(sc, g, ga, gd)
        ctx.scene = None
        return ga, gd, None, None
