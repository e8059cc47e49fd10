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
    e = H.check_energy(g["energy"], o.sum(axis=1), rel=1e-5, what="splat energy")
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
    """Workload 4 sizes (64x64 scan, 65,536 points, 512 bins of 8 ps, splat
    with 60 ps FWHM), one scene: forward on sampled scan points and the
    gradient on sampled points against the oracle."""
    from paper_2506_03747_gb300 import nlos
    params, sc_pts, _ = scenes.workload_glyph_batch(n_scenes=1)
    pts = sc_pts[0]
    g = H.gpu_forward(params, pts)
    rng = np.random.default_rng(2)
    for s in rng.choice(4096, size=4, replace=False):
        o = oracle.forward_splat(params, pts, int(s), 1)
        H.check_bins(g["tau"][s:s + 1], o, what=f"splat s={s}")
    S, B = 4096, 512
    gt = rng.normal(size=(S, B)).astype(np.float32)
    sc = nlos.scene_create(nlos.params(params), pts)
    ga = torch.empty(sc.num_points, dtype=torch.float32, device="cuda")
    gd = torch.empty(sc.num_points, dtype=torch.float32, device="cuda")
    nlos.simulate_backward(sc, torch.from_numpy(gt).cuda(), ga, gd)
    torch.cuda.synchronize()
    sel = np.sort(rng.choice(pts.shape[0], size=64, replace=False))
    oa, od = oracle.backward_splat(params, pts[sel], gt.astype(np.float64))
    a = ga.cpu().numpy()[sel]
    d = gd.cpu().numpy()[sel]
    assert np.abs(a - oa).max() <= 1e-3 * np.abs(oa).max()
    assert np.abs(d - od).max() <= 1e-3 * np.abs(od).max()


def test_autograd_function_against_finite_differences():
    from paper_2506_03747_gb300.autograd import NlosSplat
    from paper_2506_03747_gb300 import nlos
    H.lib()
    params, pts = _small(n_side=16, scan=8)
    pts[:, 6] = 0.3 + 0.7 * pts[:, 6]  # keep albedo - h >= 0 for the differences
    prm = nlos.params(params)
    P = pts.shape[0]
    points = torch.from_numpy(pts).cuda()
    albedo = torch.from_numpy(pts[:, 6].copy()).cuda().requires_grad_(True)
    depth = torch.zeros(P, device="cuda", requires_grad=True)
    target = NlosSplat.apply(albedo.detach() * 0.9, depth.detach() + 2e-3, points, prm).detach()
    loss = ((NlosSplat.apply(albedo, depth, points, prm) - target) ** 2).sum()
    loss.backward()

    def L(a, d):
        with torch.no_grad():
            return float(((NlosSplat.apply(a, d, points, prm) - target) ** 2).sum())

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
