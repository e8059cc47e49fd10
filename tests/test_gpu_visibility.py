"""GPU parity of the visibility extension (occluders, through the C ABI)
against the FP64 oracle: a union of spheres and boxes shadowing itself
(confocal and non-confocal, at a small size and on sampled transients of the
full union workload), a sphere's shadow on a plane, removal of the
occluders, and the argument checks.

Pairs whose chord lies within OCC_DELTA of the threshold may come out either
way in FP32 (near-tangent segments); their weight is an allowance, like the
weight of pairs near a bin edge."""
import numpy as np
import pytest
import torch

import oracle
import scenes
from paper_2506_03747_gb300 import nlos
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu

OCC_DELTA = 2e-3  # FP32 band of the chord (fraction of the segment)


def _gpu(params, pts, occ):
    H.lib()
    sc = nlos.scene_create(nlos.params(params), pts)
    nlos.scene_set_occluders(sc, occ)
    S, B = sc.num_scan, sc.num_bins
    tau = torch.empty((S, B), dtype=torch.float32, device="cuda")
    en = torch.empty(S, dtype=torch.float64, device="cuda")
    nlos.simulate(sc, tau, None, en)
    torch.cuda.synchronize()
    out = tau.cpu().numpy().astype(np.float64), en.cpu().numpy()
    sc.destroy()
    return out


def _check(params, pts, occ, s_begin=0, s_count=None, what=""):
    tau, en = _gpu(params, pts, occ)
    S = tau.shape[0]
    if s_count is None:
        s_count = S - s_begin
    sl = slice(s_begin, s_begin + s_count)
    B = int(params["num_bins"])
    r = oracle.forward_binned(params, pts, s_begin, s_count, eps=H.u_eps(B), occ=occ,
                              occ_delta=OCC_DELTA)
    taps = oracle.jitter_taps(params["jitter_fwhm_s"], params["bin_width_s"])
    pad = params.get("jitter_padding", "zero")
    tau_g = oracle.jitter(r["tau"], taps, pad)
    allow_raw = r["flip_mass"] + r["occ_mass"]
    allow = oracle.jitter(allow_raw, taps, pad)
    err = H.check_bins(tau[sl], tau_g, allow=allow, what=what)
    e_allow = allow_raw.sum(axis=1) + r["edge_mass"]
    H.check_energy(en[sl], tau_g.sum(axis=1), allow=e_allow, what=what)
    return err, r


def _union(n_points, seed=scenes.SEED_BASE + 2):
    rng = np.random.default_rng(seed)
    pts, prims = scenes.primitive_union_points(rng, n_points)
    return pts, scenes.occluder_records(prims)


@pytest.mark.parametrize("scan_mode,cos_mode", [("confocal", "object"),
                                                ("nonconfocal", "object"),
                                                ("confocal", "none"),
                                                ("nonconfocal", "object_wall")])
def test_union_self_shadow(scan_mode, cos_mode):
    pts, occ = _union(6000)
    params = scenes.default_params(scan_nx=20, scan_ny=13, wall_half_x=1.0, wall_half_y=1.0,
                                   scan_mode=scan_mode, laser_xy=(0.3, -0.2),
                                   bin_width_s=8e-12, num_bins=700, standoff_m=1.0,
                                   standoff_mode="euclidean", window_start_m=2.4,
                                   jitter_fwhm_s=60e-12, cos_mode=cos_mode)
    err, r = _check(params, pts, occ, what=f"union {scan_mode} {cos_mode}")
    plain = oracle.forward_binned(params, pts)["tau"]
    # the occluders do remove light, and only a few pairs sit on the threshold
    assert r["tau"].sum() < 0.999 * plain.sum()
    print(scan_mode, cos_mode, "max err/peak", err, "borderline pairs", r["n_occ_border"],
          "light kept", r["tau"].sum() / plain.sum())


def test_sphere_shadow_on_plane():
    params = scenes.default_params(scan_nx=8, scan_ny=8, wall_half_x=0.5, wall_half_y=0.5,
                                   bin_width_s=8e-12, num_bins=900, standoff_m=0.0,
                                   standoff_mode="constant", jitter_fwhm_s=30e-12)
    pts = scenes.plane_grid(96, 0.6, 1.0, 0.8)
    occ = np.array([[0, 0.05, -0.1, 0.5, 0.12, 0, 0, 0], [1, -0.4, 0.1, 0.6, -0.2, 0.3, 0.65, 0]],
                   dtype=np.float32)
    _check(params, pts, occ, what="plane shadow")


def test_removing_occluders_restores_plain():
    params, pts = scenes.workload_plane32()
    H.lib()
    sc = nlos.scene_create(nlos.params(params), pts)
    S, B = sc.num_scan, sc.num_bins
    tau = torch.empty((S, B), dtype=torch.float32, device="cuda")
    nlos.scene_set_occluders(sc, np.array([[0, 0, 0, 0.25, 0.1, 0, 0, 0]], dtype=np.float32))
    nlos.simulate(sc, tau)
    shadowed = tau.sum().item()
    nlos.scene_set_occluders(sc, None)
    nlos.simulate(sc, tau)
    torch.cuda.synchronize()
    plain = H.gpu_forward(params, pts)["tau"]
    assert np.allclose(tau.cpu().numpy(), plain, rtol=0, atol=1e-5 * plain.max())
    assert shadowed < 0.99 * plain.sum()
    sc.destroy()


def test_occluder_argument_checks():
    params, pts = scenes.workload_plane32()
    H.lib()
    sc = nlos.scene_create(nlos.params(params), pts)
    bad = [
        [[2, 0, 0, 0.5, 0.1, 0, 0, 0]],            # unknown kind
        [[0, 0, 0, 0.5, 0.0, 0, 0, 0]],            # radius 0
        [[1, 0, 0, 0.5, 0.1, 0.1, 0.4, 0]],        # box with a_z >= b_z
        [[0, np.nan, 0, 0.5, 0.1, 0, 0, 0]],       # non-finite
        [[0, 0, 0, 0.5, 0.1, 0, 0, 0]] * 17,       # too many
    ]
    for rec in bad:
        with pytest.raises(nlos.NlosError) as e:
            nlos.scene_set_occluders(sc, np.asarray(rec, dtype=np.float32))
        assert e.value.status == nlos.EINVAL
    sc.destroy()
    sp = dict(params, bin_mode="splat", jitter_fwhm_s=60e-12)
    sc = nlos.scene_create(nlos.params(sp), pts)
    nlos.scene_set_occluders(sc, np.array([[0, 0, 0, 0.25, 0.1, 0, 0, 0]], dtype=np.float32))
    tau = torch.empty((sc.num_scan, sc.num_bins), dtype=torch.float32, device="cuda")
    with pytest.raises(nlos.NlosError) as e:
        nlos.simulate(sc, tau)
    assert e.value.status == nlos.EINVAL
    sc.destroy()


def test_union64_full_size_sampled():
    """The union workload at full size (4096 scan points x 262,144 points) with
    its own primitives as occluders, in the launch configuration the benchmark
    times; 96 transients against the oracle."""
    params, _ = scenes.workload_union64()
    rng = np.random.default_rng(scenes.SEED_BASE + 2)
    pts, prims = scenes.primitive_union_points(rng, 262144)
    occ = scenes.occluder_records(prims)
    params = dict(params, noise_mode="none")
    for s0 in (0, 2048 + 17, 4096 - 32):
        err, r = _check(params, pts, occ, s_begin=s0, s_count=32, what=f"union64 occ s0={s0}")
        print("union64 occluded", s0, err, r["n_occ_border"])
