"""torch.autograd.Function around the differentiable splat forward and its
hand-written adjoint (both CUDA kernels behind the C ABI).

``NlosSplat.apply(albedo, depth, scene)`` returns tau [S, B] of ``scene`` (an
``nlos.Scene`` with bin_mode = splat, created once from the base point
records) with point p given albedo ``albedo[p]`` and displaced by ``depth[p]``
metres along its normal; gradients flow to ``albedo`` and ``depth``. The
displacement and the re-packing run on the device
(``nlos_scene_set_albedo_depth``); this wrapper only checks dtypes and
contiguity. The adjoint is evaluated at the displaced points, so it is exact
at any depth. If the scene was moved again between a forward and its
backward, the backward first puts back the forward's albedo and depth.
"""
from __future__ import annotations

import torch

from . import nlos


def _f32(t: torch.Tensor) -> torch.Tensor:
    return t.detach().to(torch.float32).contiguous()


class NlosSplat(torch.autograd.Function):
    @staticmethod
    def forward(ctx, albedo, depth, scene):
        a, d = _f32(albedo), _f32(depth)
        nlos.scene_set_albedo_depth(scene, a, d)
        tau = torch.empty((scene.num_scan, scene.num_bins), dtype=torch.float32,
                          device=a.device)
        nlos.forward(scene, tau)
        ctx.scene, ctx.version = scene, scene.version
        ctx.save_for_backward(a, d)
        return tau

    @staticmethod
    def backward(ctx, grad_tau):
        sc = ctx.scene
        a, d = ctx.saved_tensors
        if sc.version != ctx.version:
            nlos.scene_set_albedo_depth(sc, a, d)
        g = grad_tau.contiguous().to(torch.float32)
        ga = torch.empty(sc.num_points, dtype=torch.float32, device=g.device)
        gd = torch.empty(sc.num_points, dtype=torch.float32, device=g.device)
        nlos.simulate_backward(sc, g, ga, gd)
        ctx.scene = None
        return ga, gd, None
