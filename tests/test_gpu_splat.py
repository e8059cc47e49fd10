"""GPU parity of the differentiable splat forward and its hand-written adjoint
(through the C ABI) against the FP64 oracle, and the torch.autograd wrapper
against central finite differences of the GPU forward."""
import numpy as np
import pytest
import torch

import oracle
import scenes
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _small(n_side=64, scan=16, seed=0, fwhm=60e-12, **kw):
    rng = np.random.default_rng(seed)
    params = scenes.default_params(scan_nx=scan, scan_ny=scan, wall_half_x=0.5, wall_half_y=0.5,
                                   bin_width_s=8e-12, num_bins=512, jitter_fwhm_s=fwhm,
                                   bin_mode="splat", **kw)
    pts = scenes.plane_grid(n_side, 0.5, 0.5, scenes.glyph(rng, 8, n_side // 8))
    pts[:, 2] += rng.normal(0, 0.01, size=pts.shape[0]).astype(np.float32)
    return params, pts


# 60 ps FWHM at 8 ps bins is sigma = 3.2 bins (moment form), 30 ps is 1.6 bins
# (per-tap form)
@pytest.mark.parametrize("fwhm", [60e-12, 30e-12])
@pytest.mark.parametrize("scan_mode,cos_mode", [("confocal", "object"), ("confocal", "none"),
                                                ("nonconfocal", "object_wall")])
def test_splat_forward_matches_oracle(scan_mode, cos_mode, fwhm):
    params, pts = _small(scan_mode=scan_mode, cos_mode=cos_mode, laser_xy=(0.1, 0.05), fwhm=fwhm)
    g = H.gpu_forward(params, pts)
    o = oracle.forward_splat(params, pts)
    err = H.check_bins(g["tau"], o, what="splat")
    # energy within 1e-6 of the full mass of the pairs whose splat reaches the
    # window: for a transient whose window holds only the cut tails of
    # Gaussians centred beyond its edges (a scan corner here), the tails'
    # rounding is measured against the pairs' mass, as window-edge flips are
    # in the binned mode; elsewhere that mass is the transient's energy
    S, B = g["tau"].shape
    u, w = oracle.pair_table(params, pts, np.arange(S))
    sig = oracle.sigma_bins(params["jitter_fwhm_s"], params["bin_width_s"])
    reach = (u > 0.5 - 6 * sig) & (u < B - 0.5 + 6 * sig)
    mass = (w * reach).sum(axis=1)
    e_o = o.sum(axis=1)
    bad = np.abs(g["energy"] - e_o) > 1e-6 * np.maximum(e_o, mass) + 1e-300
    assert not bad.any(), (np.argwhere(bad)[:3].ravel(), g["energy"][bad][:3], e_o[bad][:3])
    e = H.check_energy(g["energy"], e_o, allow=1e-6 * np.maximum(mass - e_o, 0.0),
                       what="splat energy")
    print("splat", scan_mode, cos_mode, err, e)


def _grad_compare(params, pts, seed=0):
    from paper_2506_03747_gb300 import nlos
    H.lib()
    S = params["scan_nx"] * params["scan_ny"]
    B = params["num_bins"]
    rng = np.random.default_rng(seed)
    gt = rng.normal(size=(S, B)).astype(np.float32)
    sc = nlos.scene_create(nlos.params(params), pts)
    ga = torch.empty(sc.num_points, dtype=torch.float32, device="cuda")
    gd = torch.empty(sc.num_points, dtype=torch.float32, device="cuda")
    nlos.simulate_backward(sc, torch.from_numpy(gt).cuda(), ga, gd)
    torch.cuda.synchronize()
    oa, od = oracle.backward_splat(params, pts, gt.astype(np.float64))
    res = {}
    for name, a, b in [("albedo", ga.cpu().numpy(), oa), ("depth", gd.cpu().numpy(), od)]:
        err = np.abs(a - b).max() / np.abs(b).max()
        cos = float(np.dot(a, b) / (np.linalg.norm(a) * np.linalg.norm(b)))
        res[name] = (err, cos)
        assert err <= 1e-3, (name, err)
        assert cos > 0.9999, (name, cos)
    return res


@pytest.mark.parametrize("fwhm", [60e-12, 30e-12])
@pytest.mark.parametrize("scan_mode,cos_mode", [("confocal", "object"), ("confocal", "none"),
                                                ("nonconfocal", "object"),
                                                ("nonconfocal", "object_wall")])
def test_adjoint_matches_oracle_gradient(scan_mode, cos_mode, fwhm):
    params, pts = _small(n_side=32, scan=12, scan_mode=scan_mode, cos_mode=cos_mode,
                         laser_xy=(0.1, 0.05), standoff_m=0.3, standoff_mode="euclidean",
                         fwhm=fwhm)
    print(scan_mode, cos_mode, _grad_compare(params, pts))


def test_workload_glyph_batch_sampled():
    """Workload 4 at its sizes (8 scenes, each a 64x64 scan, 65,536 points,
    512 bins of 8 ps, splat with 60 ps FWHM): for every scene, the forward on
    sampled scan points and the gradient on sampled points against the
    oracle."""
    from paper_2506_03747_gb300 import nlos
    params, sc_pts, _ = scenes.workload_glyph_batch()
    assert len(sc_pts) == 8
    rng = np.random.default_rng(2)
    S, B = 4096, 512
    for k, pts in enumerate(sc_pts):
        g = H.gpu_forward(params, pts)
        for s in rng.choice(S, size=3, replace=False):
            o = oracle.forward_splat(params, pts, int(s), 1)
            H.check_bins(g["tau"][s:s + 1], o, what=f"scene {k} splat s={s}")
        gt = rng.normal(size=(S, B)).astype(np.float32)
        sc = nlos.scene_create(nlos.params(params), pts)
        ga = torch.empty(sc.num_points, dtype=torch.float32, device="cuda")
        gd = torch.empty(sc.num_points, dtype=torch.float32, device="cuda")
        nlos.simulate_backward(sc, torch.from_numpy(gt).cuda(), ga, gd)
        torch.cuda.synchronize()
        sel = np.sort(rng.choice(pts.shape[0], size=48, replace=False))
        oa, od = oracle.backward_splat(params, pts[sel], gt.astype(np.float64))
        a = ga.cpu().numpy()[sel]
        d = gd.cpu().numpy()[sel]
        assert np.abs(a - oa).max() <= 1e-3 * np.abs(oa).max(), k
        assert np.abs(d - od).max() <= 1e-3 * np.abs(od).max(), k
        sc.destroy()


def test_autograd_function_against_finite_differences():
    from paper_2506_03747_gb300.autograd import NlosSplat
    from paper_2506_03747_gb300 import nlos
    H.lib()
    params, pts = _small(n_side=16, scan=8)
    pts[:, 6] = 0.3 + 0.7 * pts[:, 6]  # keep albedo - h >= 0 for the differences
    P = pts.shape[0]
    scene = nlos.scene_create(nlos.params(params), torch.from_numpy(pts).cuda())
    albedo = torch.from_numpy(pts[:, 6].copy()).cuda().requires_grad_(True)
    depth = torch.zeros(P, device="cuda", requires_grad=True)
    target = NlosSplat.apply(albedo.detach() * 0.9, depth.detach() + 2e-3, scene).detach()
    loss = ((NlosSplat.apply(albedo, depth, scene) - target) ** 2).sum()
    loss.backward()

    def L(a, d):
        with torch.no_grad():
            return float(((NlosSplat.apply(a, d, scene) - target) ** 2).sum())

    rng = np.random.default_rng(4)
    for i in rng.choice(P, size=6, replace=False):
        h = 1e-2
        a1 = albedo.detach().clone(); a1[i] += h
        a0 = albedo.detach().clone(); a0[i] -= h
        fd = (L(a1, depth.detach()) - L(a0, depth.detach())) / (2 * h)
        assert albedo.grad[i].item() == pytest.approx(fd, rel=2e-2, abs=1e-6 * abs(loss.item()))
        h = 1e-4
        d1 = depth.detach().clone(); d1[i] += h
        d0 = depth.detach().clone(); d0[i] -= h
        fd = (L(albedo.detach(), d1) - L(albedo.detach(), d0)) / (2 * h)
        assert depth.grad[i].item() == pytest.approx(fd, rel=5e-2, abs=1e-4 * abs(loss.item()))


def test_autograd_config4_directional_differences():
    """NlosSplat at workload 4's size (one glyph scene: 64x64 scan, 65,536
    points, 512 bins): one scene reused across steps, and the gradient of the
    L2 loss against a perturbed target checked along random directions of
    albedo and depth by central differences of the GPU forward (FP64 loss)."""
    from paper_2506_03747_gb300.autograd import NlosSplat
    from paper_2506_03747_gb300 import nlos
    H.lib()
    params, sc_pts, tgt_pts = scenes.workload_glyph_batch(n_scenes=1)
    pts, tp = sc_pts[0], tgt_pts[0]
    P = pts.shape[0]
    scene = nlos.scene_create(nlos.params(params), torch.from_numpy(pts).cuda())
    tsc = nlos.scene_create(nlos.params(params), tp)
    target = torch.empty((scene.num_scan, scene.num_bins), dtype=torch.float32, device="cuda")
    nlos.forward(tsc, target)
    tsc.destroy()
    albedo = torch.from_numpy(pts[:, 6].copy()).cuda().requires_grad_(True)
    depth = torch.zeros(P, device="cuda", requires_grad=True)

    def loss_of(a, d):
        return ((NlosSplat.apply(a, d, scene) - target).double() ** 2).sum()

    for step in range(2):  # the scene is reused: a second step sees the same state
        albedo.grad = None
        depth.grad = None
        loss = loss_of(albedo, depth)
        loss.backward()
    rng = np.random.default_rng(9)
    lit = pts[:, 6] > 0  # albedo moves only where it stays positive (the glyph's 1s)
    for name, h in (("albedo", 1e-2), ("depth", 5e-5)):
        v = rng.normal(size=P).astype(np.float32)
        if name == "albedo":
            v[~lit] = 0.0
        v = torch.from_numpy(v).cuda()
        with torch.no_grad():
            if name == "albedo":
                lp = float(loss_of(albedo.detach() + h * v, depth.detach()))
                lm = float(loss_of(albedo.detach() - h * v, depth.detach()))
                an = float((albedo.grad.double() * v.double()).sum())
            else:
                lp = float(loss_of(albedo.detach(), depth.detach() + h * v))
                lm = float(loss_of(albedo.detach(), depth.detach() - h * v))
                an = float((depth.grad.double() * v.double()).sum())
        fd = (lp - lm) / (2 * h)
        print(name, "directional derivative: adjoint", an, "central differences", fd)
        assert an == pytest.approx(fd, rel=2e-2), name
    scene.destroy()
