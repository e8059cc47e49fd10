"""GPU parity of the forward hot path (through the C ABI) against the FP64
oracle: pair table (u, w), binned transient, fused jitter, per-transient
energy, window splitting, ragged scan and point tails, every cosine, scan and
stand-off mode, the workload sizes themselves, and degenerate inputs."""
import zlib

import numpy as np
import pytest
import torch

import oracle
import scenes
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _compare(params, pts, s_begin=0, s_count=None, exact_flips=True, threads=0,
             rel_energy=H.REL_ENERGY):
    """Full-cube (or scan-range) comparison; returns the measured errors.

    Per-transient energies are held to rel_energy (1e-6 by default); the total
    energy of the cube always to 1e-6."""
    g = H.gpu_forward(params, pts)
    S = g["tau"].shape[0]
    if s_count is None:
        s_count = S - s_begin
    sl = slice(s_begin, s_begin + s_count)
    o = H.oracle_with_allowance(params, pts, s_begin, s_count, threads=threads)
    R = (o["taps"].size - 1) // 2
    B = int(params["num_bins"])
    edge_bins = np.r_[0:R + 1, max(0, B - R - 1):B]
    allow_e = o["edge"] + o["flip"][:, edge_bins].sum(axis=1)
    res = {}
    res["bin_err"] = H.check_bins(g["tau"][sl], o["tau_g"], allow=o["flip_g"], what="tau_G")
    res["energy_err"] = H.check_energy(g["energy"][sl], o["tau_g"].sum(axis=1), allow=allow_e,
                                       rel=rel_energy, what="energy")
    e_tot_g, e_tot_o = g["energy"][sl].sum(), o["tau_g"].sum()
    res["total_energy_err"] = abs(e_tot_g - e_tot_o) / e_tot_o if e_tot_o > 0 else 0.0
    assert abs(e_tot_g - e_tot_o) <= H.REL_ENERGY * e_tot_o + allow_e.sum()
    if exact_flips:
        tau_fc, nflip, du = H.flip_corrected_oracle(params, pts, g["scene"], s_begin, s_count)
        tau_fc_g = oracle.jitter(tau_fc, o["taps"], o["pad"])
        res["bin_err_exact"] = H.check_bins(g["tau"][sl], tau_fc_g, what="tau_G (flips moved)")
        res["energy_err_exact"] = H.check_energy(g["energy"][sl], tau_fc_g.sum(axis=1),
                                                 rel=rel_energy, what="energy (flips moved)")
        res["flips"] = nflip
        res["max_du"] = du
        assert du < H.u_eps(int(params["num_bins"]))
    res["n_boundary_eps"] = o["n_boundary"]
    return res


def test_workload_plane32_full_cube():
    params, pts = scenes.workload_plane32()
    r = _compare(params, pts)
    print("plane32", r)
    assert r["bin_err_exact"] < 1e-4 and r["energy_err_exact"] < 1e-6


@pytest.mark.parametrize("scan_mode", ["confocal", "nonconfocal"])
@pytest.mark.parametrize("cos_mode", ["none", "object", "object_wall"])
@pytest.mark.parametrize("standoff_mode", ["euclidean", "constant"])
def test_modes_ragged(scan_mode, cos_mode, standoff_mode):
    """Random surface normals (some transients at grazing incidence), ragged
    scan tiles and an odd point count; every transient's energy within 1e-6."""
    rng = np.random.default_rng(zlib.crc32(f"{scan_mode}/{cos_mode}/{standoff_mode}".encode()))
    pts = scenes.random_points(rng, 1001, half=0.6)  # odd: padded pair
    params = scenes.default_params(scan_nx=33, scan_ny=17, wall_half_x=0.7, wall_half_y=0.4,
                                   scan_mode=scan_mode, laser_xy=(0.13, -0.07), cos_mode=cos_mode,
                                   standoff_m=0.35, standoff_mode=standoff_mode,
                                   bin_width_s=6e-12, num_bins=700, jitter_fwhm_s=45e-12)
    r = _compare(params, pts)
    print(scan_mode, cos_mode, standoff_mode, r)


def test_window_split_and_unaligned_bins():
    """More bins than one shared-memory window holds (two windows), with a
    bin count that is not a multiple of 4 (scalar reductions)."""
    rng = np.random.default_rng(3)
    pts = scenes.random_points(rng, 777, half=0.5, z_lo=0.2, z_hi=1.8)
    params = scenes.default_params(scan_nx=9, scan_ny=7, wall_half_x=0.5, wall_half_y=0.5,
                                   bin_width_s=2e-12, num_bins=2501, jitter_fwhm_s=30e-12,
                                   standoff_m=0.1, standoff_mode="euclidean")
    r = _compare(params, pts)
    print("window split", r)


@pytest.mark.parametrize("B", [2501, 700])
def test_replicate_padding(B):
    """Jitter with the edge bins continued outside the window: the window
    starts inside the scene (bin 0 populated) and ends inside it (the last bin
    populated), with one window (700 bins) and several (2501, not a multiple
    of 4)."""
    rng = np.random.default_rng(11)
    pts = scenes.random_points(rng, 901, half=0.5, z_lo=0.2, z_hi=1.8)
    params = scenes.default_params(scan_nx=9, scan_ny=7, wall_half_x=0.5, wall_half_y=0.5,
                                   bin_width_s=2e-12, num_bins=B, jitter_fwhm_s=30e-12,
                                   standoff_m=0.1, standoff_mode="euclidean",
                                   window_start_m=1.2, jitter_padding="replicate")
    g = H.gpu_forward(params, pts)
    assert g["tau"][:, 0].any() and g["tau"][:, -1].any()
    r = _compare(params, pts)
    print("replicate", B, r)


def test_workload_union64_full_cube():
    """Workload 2 at full size (4096 x 262144 pairs), every transient."""
    params, pts = scenes.workload_union64()
    r = _compare(params, pts, exact_flips=False)
    print("union64", r)
    # exact flip accounting on two rows through the populated centre
    s0 = 31 * 64
    r2 = _compare(params, pts, s0, 128)
    print("union64 rows 31-32", r2)
    assert r2["flips"] >= 0 and np.count_nonzero(H.gpu_forward(params, pts)["energy"]) > 500


def test_workload_heightfield128_sampled():
    """Workload 3 (128x128 non-confocal scan, 1,048,576 points, 1024 bins of
    4 ps) in the benchmark's launch configuration, checked on 256 sampled scan
    points (transients are independent of one another)."""
    params, pts = scenes.workload_heightfield128()
    g = H.gpu_forward(params, pts)
    rng = np.random.default_rng(1)
    rows = np.sort(rng.choice(128 * 128, size=256, replace=False))
    worst, worst_e, populated = 0.0, 0.0, 0
    for s in rows:
        o = H.oracle_with_allowance(params, pts, int(s), 1)
        worst = max(worst, H.check_bins(g["tau"][s:s + 1], o["tau_g"], allow=o["flip_g"],
                                        what=f"s={s}"))
        R = (o["taps"].size - 1) // 2
        allow_e = o["edge"] + o["flip"][:, np.r_[0:R + 1, 1024 - R - 1:1024]].sum(axis=1)
        worst_e = max(worst_e, H.check_energy(g["energy"][s:s + 1], o["tau_g"].sum(axis=1),
                                              allow=allow_e, what=f"energy s={s}"))
        populated += int(o["tau"].sum() > 0)
    print("heightfield128 worst rel bin err", worst, "energy", worst_e, "populated", populated)
    assert populated >= 100


def test_empty_and_degenerate():
    H.lib()
    from paper_2506_03747_gb300 import nlos
    # no points: zero transient
    params = scenes.default_params(scan_nx=5, scan_ny=3, num_bins=64)
    g = H.gpu_forward(params, np.zeros((0, 8), dtype=np.float32))
    assert (g["tau"] == 0).all() and (g["energy"] == 0).all()
    # one scan point, one point, one bin: impulse lands in bin 0 or nowhere
    pt = scenes.single_point(0.0, 0.0, 0.5)
    p1 = scenes.default_params(scan_nx=1, scan_ny=1, wall_half_x=0.01, wall_half_y=0.01,
                               num_bins=1, bin_width_s=16e-12, window_start_m=0.999)
    g = H.gpu_forward(p1, pt)
    o = oracle.forward_binned(p1, pt)["tau"]
    np.testing.assert_allclose(g["tau"], o, rtol=1e-5)
    assert o.sum() > 0
    # everything outside the window
    p2 = dict(p1, window_start_m=5.0)
    assert (H.gpu_forward(p2, pt)["tau"] == 0).all()
    # invalid inputs are rejected on the host or by the packing kernel's checks
    bad = pt.copy()
    bad[0, 2] = -0.1
    with pytest.raises(nlos.NlosError):
        nlos.scene_create(nlos.params(p1), bad)
    with pytest.raises(nlos.NlosError):
        nlos.scene_create(nlos.params(p1, num_bins=0), pt)
    with pytest.raises(nlos.NlosError):
        nlos.scene_create(nlos.params(p1, bin_width_s=-1.0), pt)


def test_boundary_pair_count_matches_oracle():
    """The kernel's count of pairs within eps of a bin edge (FP32 u) against the
    oracle's (FP64 u): equal up to pairs whose distance to the edge is itself
    within the FP32 error of eps."""
    params, pts = scenes.workload_plane32()
    for eps in (1e-3, 1e-2):
        g = H.gpu_forward(params, pts, stats=True, boundary_eps=eps)
        o = oracle.forward_binned(params, pts, eps=eps)
        n_g, n_o = g["stats"]["boundary_pairs"], o["n_boundary"]
        lo = oracle.forward_binned(params, pts, eps=eps - H.U_EPS / 2)["n_boundary"]
        hi = oracle.forward_binned(params, pts, eps=eps + H.U_EPS / 2)["n_boundary"]
        print("boundary pairs", eps, n_g, n_o, (lo, hi))
        assert lo <= n_g <= hi
    # At eps = 1e-6 bin the FP32 u (ulp ~ 1e-5 bin at u ~ 200) cannot resolve
    # the distance to the edge, so the kernel's count is bounded by the
    # oracle's counts at eps +- U_EPS/2; the flips that actually happen are
    # counted exactly (GPU bin against FP64 bin, pair by pair), and each one
    # is a pair within U_EPS of an edge.
    g = H.gpu_forward(params, pts, stats=True, boundary_eps=1e-6)
    n_g = g["stats"]["boundary_pairs"]
    n_o = oracle.forward_binned(params, pts, eps=1e-6)["n_boundary"]
    hi = oracle.forward_binned(params, pts, eps=1e-6 + H.U_EPS / 2)["n_boundary"]
    assert 0 <= n_g <= hi
    _, nflip, du = H.flip_corrected_oracle(params, pts, g["scene"], 0, g["tau"].shape[0])
    # a pair can only flip if its distance to an edge is below |u32 - u64|
    assert du < H.U_EPS
    assert nflip <= oracle.forward_binned(params, pts, eps=du * (1 + 1e-9))["n_boundary"]
    print("pairs within 1e-6 bin of an edge: gpu (fp32 u)", n_g, "oracle (fp64 u)", n_o,
          "bound", hi, "; bins that flipped", nflip)


def test_u_precision_all_workloads():
    """max |u_fp32 - u_fp64| over sampled pairs of every workload: the FP32
    bin coordinate (path lengths taken relative to the window start) stays
    well below 1e-3 bin."""
    cases = [scenes.workload_plane32(), scenes.workload_union64(), scenes.workload_heightfield128()]
    for params, pts in cases:
        g = H.gpu_forward(params, pts[: min(len(pts), 20000)], energy=False)
        S = g["tau"].shape[0]
        ids = np.linspace(0, S - 1, 16).astype(int)
        worst = 0.0
        for s in ids:
            u32, _ = H.gpu_pair_table(g["scene"], int(s), 1)
            u64, _ = oracle.pair_table(params, pts[: min(len(pts), 20000)], [int(s)])
            worst = max(worst, float(np.abs(u32.astype(np.float64) - u64).max()))
        print("max |u32 - u64| (bins):", params["num_bins"], params["bin_width_s"], worst)
        assert worst < H.U_EPS


def test_paper_dataset_shape():
    """The paper's dataset configuration (Simulation section; golden fixture):
    128x128 scan over 2 m x 2 m, 1024 bins of 32 ps, 70 ps FWHM jitter (k = 5),
    albedo 1, on a 128x128 depth-map-like heightfield; sampled transients
    against the oracle."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_dataset_params.json")) as f:
        gd = json.load(f)
    rng = np.random.default_rng(77)
    pts = scenes.heightfield_points(rng, gd["scan_side"])
    pts[:, 6] = gd["albedo"]
    n = gd["scan_side"]
    params = scenes.default_params(scan_nx=n, scan_ny=n, wall_half_x=gd["scan_extent_m"] / 2,
                                   wall_half_y=gd["scan_extent_m"] / 2,
                                   bin_width_s=gd["bin_width_s"], num_bins=gd["num_bins"],
                                   jitter_fwhm_s=gd["jitter_fwhm_s"])
    assert oracle.jitter_taps(params["jitter_fwhm_s"], params["bin_width_s"]).size == 5
    g = H.gpu_forward(params, pts)
    rows = np.sort(rng.choice(n * n, size=96, replace=False))
    worst = 0.0
    for s in rows:
        o = H.oracle_with_allowance(params, pts, int(s), 1)
        worst = max(worst, H.check_bins(g["tau"][s:s + 1], o["tau_g"], allow=o["flip_g"],
                                        what=f"s={s}"))
        R = (o["taps"].size - 1) // 2
        B = params["num_bins"]
        allow_e = o["edge"] + o["flip"][:, np.r_[0:R + 1, B - R - 1:B]].sum(axis=1)
        H.check_energy(g["energy"][s:s + 1], o["tau_g"].sum(axis=1), allow=allow_e,
                       what=f"energy s={s}")
    print("paper dataset shape: worst rel bin err", worst)


def test_early_out_count():
    """The forward rules out (tile, block) units from their bounds and skips
    (warp, point pair) groups that no lane can bin; it reports the pairs of the
    units it staged and the pairs it evaluated in full: multiples of 64, within
    the padded pair count, and zero when the window lies beyond every path."""
    params, pts = scenes.workload_union64()
    g = H.gpu_forward(params, pts, stats=True)
    full, tested = g["stats"]["pairs_full"], g["stats"]["pairs_tested"]
    S, P = g["tau"].shape[0], pts.shape[0]
    assert full % 64 == 0 and tested % 64 == 0
    assert 0 < full <= tested <= ((S + 31) // 32 * 32) * ((P + 1) // 2 * 2)
    print("union64 pairs evaluated in full:", full / (S * P), "in staged units:", tested / (S * P))
    far = dict(params, window_start_m=100.0)
    g2 = H.gpu_forward(far, pts, stats=True)
    # every unit is ruled out from the bounds: no pair is touched
    assert g2["stats"]["pairs_full"] == 0 and g2["stats"]["pairs_tested"] == 0
    assert not g2["tau"].any()


def test_measured_peaks_plausible():
    """The roofline denominators of nlos_measure_peaks: every rate positive and
    below the part's issue limits per SM clock (128 FP32 lanes, 16 MUFU lanes,
    32 shared-memory lanes); FP64 fma below FP32; a shared reduction with a
    quarter of the lanes active no faster per lane than four times a full one."""
    H.lib()
    from paper_2506_03747_gb300 import nlos
    p = nlos.measure_peaks()
    assert p["num_sms"] > 0
    assert 0 < p["ffma"] <= 128.5 and 0 < p["ffma2"] <= 257
    for k in ("sqrt_approx", "rcp_approx", "rsqrt_approx"):
        assert 0 < p[k] <= 16.5
    for k in ("red_f32", "red_u32", "red_u64", "rmw_f32", "red_f32_quarter", "red_u32_quarter"):
        assert 0 < p[k] <= 32.5
    assert 0 < p["dfma"] < p["ffma"]
    assert p["red_f32_quarter"] <= 4 * p["red_f32"] * 1.05
