"""Pins of the FP64 CPU oracle against facts fixed by the paper and by
mathematics, independent of the oracle's own code: closed forms of Eq. 1 for a
single point and for a fronto-parallel plane, invariants (energy, linearity,
symmetry, translation), a 50-digit brute force, library routines (scipy's
Gaussian filter and normal pdf, curand's host Philox4x32-10 generator) and the
Poisson distribution itself.
"""
import ctypes
import ctypes.util
import json
import math
import os

import numpy as np
import pytest

import oracle
import scenes

C = 299792458.0
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _params(**kw):
    return scenes.default_params(**kw)


# ---------------------------------------------------------------------------
# Eq. 1, single point: a point facing the wall straight below a confocal scan
# spot at depth d returns all of its light at path 2d, with weight
# rho * a * cos * cos / d^4 = rho * a / d^4.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("cos_mode", ["none", "object", "object_wall"])
@pytest.mark.parametrize("d", [0.3137, 0.5, 0.77731])
def test_single_point_impulse(cos_mode, d):
    p = _params(scan_nx=4, scan_ny=4, wall_half_x=0.5, wall_half_y=0.5, bin_width_s=16e-12,
                num_bins=512, cos_mode=cos_mode)
    l, _, _ = oracle.scan_geometry(p, 5)  # ix=1, iy=1 -> (-0.125, -0.125)
    assert np.allclose(l, [-0.125, -0.125, 0.0])
    pt = scenes.single_point(l[0], l[1], d, albedo=0.7, area=2e-3)
    tau = oracle.forward_binned(p, pt, 5, 1)["tau"][0]
    pt64 = pt[0].astype(np.float64)
    dd = pt64[2]
    b = math.floor(2 * dd / (C * 16e-12))
    nz = np.flatnonzero(tau)
    assert list(nz) == [b]
    expect = float(pt64[6]) * float(pt64[7]) / dd ** 4
    assert tau[b] == pytest.approx(expect, rel=1e-13)


def test_single_point_standoff_euclidean():
    """Stand-off legs |D - l| + |d - D| with D = (0, 0, h) and the window start at
    2h: the impulse moves to u = (2 sqrt(h^2 + |l|^2) - 2h + 2 d) / (c dt)."""
    h = 1.25
    p = _params(scan_nx=8, scan_ny=8, wall_half_x=1.0, wall_half_y=1.0, bin_width_s=8e-12,
                num_bins=1024, standoff_m=h, standoff_mode="euclidean")
    s = 8 * 6 + 1
    l, _, legs = oracle.scan_geometry(p, s)
    assert legs == pytest.approx(2 * math.sqrt(h * h + l[0] ** 2 + l[1] ** 2), rel=1e-15)
    pt = scenes.single_point(l[0], l[1], 0.6)
    u, w = oracle.pair(p, s, pt[0])
    dd = float(pt[0, 2])
    assert u == pytest.approx((legs - 2 * h + 2 * dd) / (C * 8e-12), rel=1e-14)
    assert w == pytest.approx(1.0 / dd ** 4, rel=1e-14)
    # constant mode: the legs do not depend on the spot
    pc = dict(p, standoff_mode="constant")
    u2, _ = oracle.pair(pc, s, pt[0])
    assert u2 == pytest.approx(2 * dd / (C * 8e-12), rel=1e-14)


def test_nonconfocal_pythagorean_point():
    """Laser at the origin, detector spot at (0.6, 0, 0), point at (0.3, 0, 0.4)
    facing the wall: both legs are 0.5 m (3-4-5 triangles), both object cosines
    are 0.8, both wall cosines are 0.8."""
    # detector spot (0.6, 0): 2x1 grid over [-1.2, 1.2] x [-0.5, 0.5]: x = -0.6, 0.6
    p = _params(scan_nx=2, scan_ny=1, wall_half_x=1.2, wall_half_y=0.5, scan_mode="nonconfocal",
                laser_xy=(0.0, 0.0), bin_width_s=4e-12, num_bins=2048, standoff_m=0.0)
    l, d, _ = oracle.scan_geometry(p, 1)
    assert np.allclose(d, [0.6, 0.0, 0.0], atol=1e-15) and np.allclose(l, 0.0)
    pt = np.array([[0.3, 0.0, 0.4, 0.0, 0.0, -1.0, 1.0, 1.0]])
    for mode, fac in [("none", 1.0), ("object", 0.64), ("object_wall", 0.64 * 0.64)]:
        u, w = oracle.pair(dict(p, cos_mode=mode), 1, pt[0])
        assert u == pytest.approx(1.0 / (C * 4e-12), rel=1e-14)
        assert w == pytest.approx(fac / (0.25 * 0.25), rel=1e-13)


def test_back_facing_point_gives_no_light():
    p = _params(scan_nx=1, scan_ny=1, wall_half_x=0.1, wall_half_y=0.1)
    pt = scenes.single_point(0.0, 0.0, 0.5, normal=(0.0, 0.0, 1.0))
    assert oracle.forward_binned(p, pt)["tau"].sum() == 0.0
    pn = dict(p, cos_mode="none")
    assert oracle.forward_binned(pn, pt)["tau"].sum() > 0.0


# ---------------------------------------------------------------------------
# Eq. 1, fronto-parallel plane: onset of the light cone and the dense-sampling
# limit of the per-bin energy of a uniform plane at depth z0 (confocal):
#   with cosines: (pi rho z0^2 / 2) (r_lo^-4 - r_hi^-4),
#   without:      pi rho (r_lo^-2 - r_hi^-2),
# with r_lo = max(z0, (L0 + b c dt)/2), r_hi = (L0 + (b+1) c dt)/2.
# ---------------------------------------------------------------------------
def test_plane_onset_bin_workload_plane32():
    params, pts = scenes.workload_plane32()
    tau = oracle.forward_binned(params, pts)["tau"]
    first = np.array([np.flatnonzero(t)[0] for t in tau if t.any()])
    # every spot sits above the plane (plane spans the whole scan area), so the
    # first non-empty bin is floor(2 z0 / (c dt)) = floor(208.48) = 208 wherever the
    # albedo below the spot is non-zero; nowhere can light arrive earlier.
    assert first.min() == math.floor(2 * 0.5 / (C * 16e-12)) == 208
    assert (first >= 208).all()


@pytest.mark.parametrize("cos_mode", ["object", "none"])
def test_plane_profile_dense_limit(cos_mode):
    # 64 ps bins (19 mm of path) keep several lattice rows per annulus
    z0, rho, dt, B = 0.5, 0.8, 64e-12, 220
    p = _params(scan_nx=1, scan_ny=1, wall_half_x=0.01, wall_half_y=0.01, bin_width_s=dt,
                num_bins=B, cos_mode=cos_mode)
    cdt = C * dt
    half = 2.0
    errs = []
    for n in (500, 1000, 2000):
        pts = scenes.plane_grid(n, half, z0, rho)
        tau = oracle.forward_binned(p, pts)["tau"][0]
        b = np.arange(B)
        r_lo = np.maximum(z0, b * cdt / 2)
        r_hi = (b + 1) * cdt / 2
        ok = (r_hi > z0) & (r_hi < half)  # bins whose annulus lies inside the plane
        if cos_mode == "object":
            ref = (math.pi * rho * z0 ** 2 / 2) * (r_lo ** -4 - r_hi ** -4)
        else:
            ref = math.pi * rho * (r_lo ** -2 - r_hi ** -2)
        ref = np.where(r_hi > z0, ref, 0.0)
        # the plane's float32 albedo: compare against the rounded value
        ref *= float(np.float32(rho)) / rho * float(pts[0, 7]) / (2 * half / n) ** 2
        errs.append(np.max(np.abs(tau[ok] - ref[ok])) / ref[ok].max())
        assert (tau[~ok & (r_hi <= z0)] == 0).all()
    assert errs[-1] < 5e-3
    assert errs[0] > errs[1] > errs[2]
    if cos_mode == "object":
        # an infinite plane returns pi rho / (2 z0^2) in total; a disc of lateral
        # radius R returns that times 1 - (z0 / sqrt(R^2 + z0^2))^4, and the square
        # of half side 2 lies between the discs R = 2 and R = 2 sqrt(2)
        inf = math.pi * float(np.float32(rho)) / (2 * z0 ** 2)
        lo = inf * (1 - (z0 / math.sqrt(4 + z0 ** 2)) ** 4)
        hi = inf * (1 - (z0 / math.sqrt(8 + z0 ** 2)) ** 4)
        assert lo * (1 - 1e-3) < tau.sum() < hi * (1 + 1e-3)


# ---------------------------------------------------------------------------
# Energy and window invariants.
# ---------------------------------------------------------------------------
def test_energy_equals_sum_of_in_window_weights():
    rng = np.random.default_rng(7)
    pts = scenes.random_points(rng, 300)
    p = _params(scan_nx=5, scan_ny=4, wall_half_x=0.5, wall_half_y=0.4, bin_width_s=8e-12,
                num_bins=300, standoff_m=0.3, standoff_mode="euclidean", window_start_m=0.9)
    tau = oracle.forward_binned(p, pts)["tau"]
    u, w = oracle.pair_table(p, pts, np.arange(20))
    inwin = (u >= 0) & (u < 300)
    assert 0 < inwin.sum() < inwin.size  # some pairs fall outside the window
    np.testing.assert_allclose(tau.sum(axis=1), np.where(inwin, w, 0).sum(axis=1), rtol=1e-13)
    # every in-window pair lands in floor(u)
    for i in range(3):
        h = np.zeros(300)
        np.add.at(h, np.floor(u[i][inwin[i]]).astype(int), w[i][inwin[i]])
        np.testing.assert_allclose(tau[i], h, rtol=1e-12, atol=0)


def test_boundary_mass_accounting():
    rng = np.random.default_rng(11)
    pts = scenes.random_points(rng, 500)
    p = _params(scan_nx=3, scan_ny=3, wall_half_x=0.5, wall_half_y=0.5, bin_width_s=8e-12,
                num_bins=400)
    eps = 0.05
    r = oracle.forward_binned(p, pts, eps=eps)
    u, w = oracle.pair_table(p, pts, np.arange(9))
    m = np.floor(u + 0.5)
    near = (np.abs(u - m) < eps) & (m >= 0) & (m <= 400)
    assert r["n_boundary"] == near.sum() > 0
    edge = np.where(near & ((m == 0) | (m == 400)), w, 0).sum(axis=1)
    np.testing.assert_allclose(r["edge_mass"], edge, rtol=1e-12)
    # each near-boundary pair adds its weight to the two bins beside its edge
    assert r["flip_mass"].sum() == pytest.approx(
        (np.where(near & (m >= 1), w, 0) + np.where(near & (m < 400), w, 0)).sum(), rel=1e-12)


# ---------------------------------------------------------------------------
# Jitter (Eq. 16/17): kernel length, normalisation, symmetry, impulse response,
# and scipy's Gaussian filter with the same radius and zero padding.
# ---------------------------------------------------------------------------
def test_jitter_kernel_length_rule():
    with open(os.path.join(GOLDEN, "paper_dataset_params.json")) as f:
        g = json.load(f)
    # the paper's dataset: 70 ps FWHM at 32 ps bins -> sigma = 0.92895 bins, k = 5
    taps = oracle.jitter_taps(g["jitter_fwhm_s"], g["bin_width_s"])
    sg = g["jitter_fwhm_s"] / (2 * math.sqrt(2 * math.log(2))) / g["bin_width_s"]
    assert sg == pytest.approx(0.928946, abs=1e-6)
    assert taps.size == 2 * math.ceil(2 * sg) + 1 == 5
    # workloads 2 and 3: 60 ps / 8 ps and 30 ps / 4 ps -> sigma = 3.18496, k = 15
    for fwhm, dt in [(60e-12, 8e-12), (30e-12, 4e-12)]:
        t = oracle.jitter_taps(fwhm, dt)
        assert t.size == 15
        assert oracle.sigma_bins(fwhm, dt) == pytest.approx(3.18496, abs=1e-5)
    assert oracle.jitter_taps(0.0, 8e-12).tolist() == [1.0]


def test_jitter_taps_and_scipy():
    scipy_nd = pytest.importorskip("scipy.ndimage")
    fwhm, dt = 60e-12, 8e-12
    taps = oracle.jitter_taps(fwhm, dt)
    R = (taps.size - 1) // 2
    assert taps.sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(taps, taps[::-1], rtol=0, atol=0)
    imp = np.zeros((1, 64))
    imp[0, 30] = 1.0
    out = oracle.jitter(imp, taps)[0]
    np.testing.assert_allclose(out[30 - R:30 + R + 1], taps, rtol=1e-15)
    assert out.sum() == pytest.approx(1.0, abs=1e-15)
    rng = np.random.default_rng(3)
    x = rng.random((6, 200))
    sg = oracle.sigma_bins(fwhm, dt)
    ref = scipy_nd.gaussian_filter1d(x, sg, axis=1, mode="constant", cval=0.0, truncate=R / sg)
    np.testing.assert_allclose(oracle.jitter(x, taps), ref, rtol=1e-12, atol=1e-15)


def test_jitter_replicate_padding():
    """Replicate padding (the edge bins continue outside the window): a constant
    transient is unchanged, an edge impulse keeps the taps that fall outside,
    and scipy's 'nearest' mode with the same radius agrees."""
    scipy_nd = pytest.importorskip("scipy.ndimage")
    fwhm, dt = 70e-12, 8e-12
    taps = oracle.jitter_taps(fwhm, dt)
    R = (taps.size - 1) // 2
    const = np.full((2, 40), 3.25)
    np.testing.assert_allclose(oracle.jitter(const, taps, "replicate"), const, rtol=1e-15)
    imp = np.zeros((1, 40))
    imp[0, 0] = 1.0
    out = oracle.jitter(imp, taps, "replicate")[0]
    # bin b receives taps j >= b (sources b - j <= 0 all read bin 0)
    np.testing.assert_allclose(out[:R + 1], [taps[R + b:].sum() for b in range(R + 1)],
                               rtol=1e-14)
    # total: tap j (0 <= j <= R) reaches bins 0..j
    assert out.sum() == pytest.approx(taps[R:] @ (np.arange(R + 1) + 1.0), rel=1e-14)
    rng = np.random.default_rng(4)
    x = rng.random((5, 150))
    sg = oracle.sigma_bins(fwhm, dt)
    ref = scipy_nd.gaussian_filter1d(x, sg, axis=1, mode="nearest", truncate=R / sg)
    np.testing.assert_allclose(oracle.jitter(x, taps, "replicate"), ref, rtol=1e-12, atol=1e-15)
    # zero padding differs only within R of the edges
    z = oracle.jitter(x, taps)
    np.testing.assert_array_equal(z[:, R:-R], oracle.jitter(x, taps, "replicate")[:, R:-R])


def test_jitter_energy_leak_at_window_edges():
    taps = oracle.jitter_taps(60e-12, 8e-12)
    R = (taps.size - 1) // 2
    x = np.zeros((1, 100))
    x[0, 2] = 1.0   # within R of the start: part of the blur leaves the window
    x[0, 50] = 2.0  # far from both edges: conserved
    out = oracle.jitter(x, taps)
    leak = taps[R + 3:].sum()  # taps landing at bins < 0 (offsets -R..-3)
    assert out.sum() == pytest.approx(3.0 - leak, rel=1e-14)


# ---------------------------------------------------------------------------
# Linearity, superposition and symmetry of the transient.
# ---------------------------------------------------------------------------
def test_linearity_superposition_mirror():
    rng = np.random.default_rng(5)
    pts = scenes.random_points(rng, 200, half=0.4)
    p = _params(scan_nx=6, scan_ny=6, wall_half_x=0.5, wall_half_y=0.5, bin_width_s=8e-12,
                num_bins=500, standoff_m=0.5)
    t = oracle.forward_binned(p, pts)["tau"]
    p2 = pts.copy()
    p2[:, 6] *= 2.0
    np.testing.assert_allclose(oracle.forward_binned(p, p2)["tau"], 2 * t, rtol=1e-14)
    ta = oracle.forward_binned(p, pts[:90])["tau"]
    tb = oracle.forward_binned(p, pts[90:])["tau"]
    np.testing.assert_allclose(ta + tb, t, rtol=1e-12, atol=1e-14 * t.max())
    # mirror x -> -x of scene (positions and normals): transients mirror in ix
    m = pts.copy()
    m[:, 0] *= -1
    m[:, 3] *= -1
    tm = oracle.forward_binned(p, m)["tau"].reshape(6, 6, -1)
    np.testing.assert_allclose(tm[:, ::-1, :], t.reshape(6, 6, -1), rtol=1e-9, atol=1e-12 * t.max())


def test_nonconfocal_with_laser_on_spot_equals_confocal():
    rng = np.random.default_rng(9)
    pts = scenes.random_points(rng, 150)
    pc = _params(scan_nx=4, scan_ny=4, wall_half_x=0.4, wall_half_y=0.4, bin_width_s=4e-12,
                 num_bins=1024, standoff_m=0.7, standoff_mode="euclidean")
    s = 6
    _, d, _ = oracle.scan_geometry(pc, s)
    pn = dict(pc, scan_mode="nonconfocal", laser_xy=(float(d[0]), float(d[1])))
    for mode in ["none", "object", "object_wall"]:
        a = oracle.forward_binned(dict(pc, cos_mode=mode), pts, s, 1)["tau"]
        b = oracle.forward_binned(dict(pn, cos_mode=mode), pts, s, 1)["tau"]
        np.testing.assert_array_equal(a, b)


def test_translation_by_one_scan_cell():
    """With constant stand-off legs, shifting the scene by one scan-cell pitch in x
    moves every transient one spot in x."""
    rng = np.random.default_rng(13)
    pts = scenes.random_points(rng, 120, half=0.3).astype(np.float64)
    p = _params(scan_nx=8, scan_ny=3, wall_half_x=0.8, wall_half_y=0.3, bin_width_s=8e-12,
                num_bins=600, standoff_m=0.5, standoff_mode="constant")
    pitch = 2 * 0.8 / 8
    t0 = oracle.forward_binned(p, pts)["tau"].reshape(3, 8, -1)
    sh = pts.copy()
    sh[:, 0] += pitch
    t1 = oracle.forward_binned(p, sh)["tau"].reshape(3, 8, -1)
    np.testing.assert_allclose(t1[:, 1:, :], t0[:, :-1, :], rtol=1e-9, atol=1e-12 * t0.max())


# ---------------------------------------------------------------------------
# 50-digit brute force on a tiny grid: exact bins; weights to FP64 rounding.
# ---------------------------------------------------------------------------
def test_bruteforce_decimal_tiny():
    from tests.bruteforce_decimal import bruteforce_pairs
    rng = np.random.default_rng(17)
    pts = scenes.random_points(rng, 64, half=0.5)
    for mode, sc in [("object", "confocal"), ("object_wall", "nonconfocal"), ("none", "confocal")]:
        p = _params(scan_nx=4, scan_ny=4, wall_half_x=0.5, wall_half_y=0.5, bin_width_s=8e-12,
                    num_bins=32, standoff_m=0.4, standoff_mode="euclidean", scan_mode=sc,
                    laser_xy=(0.1, -0.2),
                    cos_mode=mode, window_start_m=1.2)
        u_ref, w_ref = bruteforce_pairs(p, pts)
        u, w = oracle.pair_table(p, pts, np.arange(16))
        np.testing.assert_allclose(u, u_ref, rtol=0, atol=1e-11)
        # FP64 weights agree to ~1e-15 except near grazing incidence, where the
        # cosine's dot product cancels (relative error ~ eps / cos)
        np.testing.assert_allclose(w, w_ref, rtol=1e-13, atol=1e-300)
        assert np.median(np.abs(w - w_ref)[w_ref > 0] / w_ref[w_ref > 0]) < 1e-15
        assert (np.floor(u) == np.floor(u_ref)).all()
        tau = oracle.forward_binned(p, pts)["tau"]
        ref = np.zeros_like(tau)
        for s in range(16):
            for q in range(64):
                if 0 <= u_ref[s, q] < 32:
                    ref[s, int(np.floor(u_ref[s, q]))] += w_ref[s, q]
        np.testing.assert_allclose(tau, ref, rtol=1e-14, atol=1e-300)


# ---------------------------------------------------------------------------
# Philox4x32-10 against curand's host generator (a separate implementation of
# Salmon et al. 2011): its stream for a seed is the blocks of counter
# (0, 0, i, 0) under key (seed_lo, seed_hi).
# ---------------------------------------------------------------------------
def _curand():
    for name in ("libcurand.so", "libcurand.so.10"):
        for d in ("/usr/local/cuda/lib64", "/usr/local/cuda/targets/sbsa-linux/lib",
                  "/usr/local/cuda/targets/x86_64-linux/lib", ""):
            try:
                return ctypes.CDLL(os.path.join(d, name) if d else name)
            except OSError:
                continue
    return None


@pytest.mark.parametrize("seed", [0, 1, 0x4E4C4F53, 0x123456789ABCDEF0, 2**64 - 1])
def test_philox_matches_curand_host_generator(seed):
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        n = 4 * 4096
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n)) == 0
        ctr = np.zeros((n // 4, 4), dtype=np.uint32)
        ctr[:, 2] = np.arange(n // 4)
        key = (seed & 0xFFFFFFFF, seed >> 32)
        np.testing.assert_array_equal(oracle.philox(ctr, key).ravel(), out)
    finally:
        lib.curandDestroyGenerator(gen)


def test_philox_avalanche():
    """Flipping one input bit flips about half of the 128 output bits."""
    rng = np.random.default_rng(1)
    flips = []
    for _ in range(200):
        c = rng.integers(0, 2**32, size=4, dtype=np.uint64).astype(np.uint32)
        k = rng.integers(0, 2**32, size=2, dtype=np.uint64).astype(np.uint32)
        bit = int(rng.integers(0, 128))
        c2 = c.copy()
        c2[bit // 32] ^= np.uint32(1 << (bit % 32))
        a = oracle.philox(c, k)[0]
        b = oracle.philox(c2, k)[0]
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    assert 60 < np.mean(flips) < 68


# ---------------------------------------------------------------------------
# Poisson sampler (Eq. 18/19): mean, variance and the full pmf (chi-square)
# against the Poisson distribution, for the inversion (lambda < 30), split
# (30 <= lambda < 150) and PTRS (lambda >= 150) branches.
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("lam", [1e-3, 0.5, 3.0, 9.9, 27.5, 29.9, 30.0, 100.0, 1500.0])
def test_poisson_sampler_distribution(lam):
    stats = pytest.importorskip("scipy.stats")
    n = 200_000
    x = oracle.poisson(np.full(n, lam, dtype=np.float32), index_base=12345, seed=99,
                       stream_tag=3).astype(np.float64)
    lam32 = float(np.float32(lam))
    se = math.sqrt(lam32 / n)
    assert abs(x.mean() - lam32) < 5 * se
    # variance: standard error of the sample variance ~ sqrt((2 lam^2 + lam) / n)
    assert abs(x.var() - lam32) < 5 * math.sqrt((2 * lam32 ** 2 + lam32) / n)
    lo, hi = stats.poisson.ppf([1e-4, 1 - 1e-4], lam32)
    edges = np.arange(int(lo), int(hi) + 2)
    obs = np.array([(x < edges[1]).sum()] + [(x == k).sum() for k in edges[1:-2]] +
                   [(x >= edges[-2]).sum()])
    pmf = np.concatenate([[stats.poisson.cdf(edges[0], lam32)],
                          stats.poisson.pmf(edges[1:-2], lam32),
                          [stats.poisson.sf(edges[-2] - 1, lam32)]])
    keep = pmf * n >= 20
    e = pmf[keep] / pmf[keep].sum() * obs[keep].sum()
    chi2 = ((obs[keep] - e) ** 2 / e).sum()
    dof = max(1, keep.sum() - 1)
    assert stats.chi2.sf(chi2, dof) > 1e-4


def test_poisson_first_draw_layout():
    """Bin i's first uniform is word (i mod 4) of the Philox block at counter
    (i // 4, 0, tag) (words from the generator pinned above): for lambda < 30
    the count is 0 exactly when u <= p0 = exp(-lambda) and at most 1 exactly
    when u <= p0 (1 + lambda), bin by bin on an unaligned range (a decision
    within 4 ulp of a threshold is skipped: expf may round either way)."""
    n, base, seed, tag = 8192, 4 * 1000 + 2, 0x1234_5678_9ABC, 5
    for lam in (0.05, 0.7, 3.0):
        x = oracle.poisson(np.full(n, lam, dtype=np.float32), base, seed, tag)
        idx = base + np.arange(n, dtype=np.uint64)
        g = idx >> np.uint64(2)
        ctr = np.stack([g & np.uint64(0xFFFFFFFF), g >> np.uint64(32), np.zeros(n, np.uint64),
                        np.full(n, tag, np.uint64)], axis=1).astype(np.uint32)
        words = oracle.philox(ctr, (seed & 0xFFFFFFFF, seed >> 32))
        w = words[np.arange(n), (idx & np.uint64(3)).astype(np.int64)]
        u = ((w >> 9).astype(np.float64) + 0.5) * 2.0 ** -23
        p0 = math.exp(-float(np.float32(lam)))
        f1 = p0 * (1.0 + float(np.float32(lam)))
        tol = 4 * 2.0 ** -24
        far0, far1 = np.abs(u - p0) > tol, np.abs(u - f1) > tol
        assert far0.mean() > 0.99 and far1.mean() > 0.99
        np.testing.assert_array_equal((x == 0)[far0], (u <= p0)[far0])
        np.testing.assert_array_equal((x <= 1)[far1], (u <= f1)[far1])


def test_poisson_dark_only_zero_probability_and_streams():
    n = 400_000
    x = oracle.poisson(np.full(n, 1e-3, dtype=np.float32), 0, 5, 0)
    p0 = (x == 0).mean()
    assert abs(p0 - math.exp(-1e-3)) < 5 * math.sqrt(math.exp(-1e-3) * (1 - math.exp(-1e-3)) / n)
    # distinct seeds / tags / indices give distinct streams; zero lambda gives 0
    a = oracle.poisson(np.full(1000, 50.0, dtype=np.float32), 0, 5, 0)
    b = oracle.poisson(np.full(1000, 50.0, dtype=np.float32), 0, 6, 0)
    c = oracle.poisson(np.full(1000, 50.0, dtype=np.float32), 0, 5, 1)
    assert (a != b).mean() > 0.9 and (a != c).mean() > 0.9
    assert oracle.poisson(np.zeros(10, dtype=np.float32), 0, 1, 0).sum() == 0
    assert oracle.poisson_one(50.0, 77, 5, 0) == a[77]


# ---------------------------------------------------------------------------
# Noise scale (Eq. 18/19, Algorithm 1 step 2.4) on a hand-worked 2 x 3 cube:
#   tau_G = [[0, 1, 2], [4, 0.5, 3]], sum 10.5, mean 1.75.
# PEAK: the maximum over the whole cube is 4 (per-transient maxima would be 2
# and 4), so with 100 photons the scale is 25 and lambda = 25 tau_G + dark.
# PAPER_NR: the squared deviations from 1.75 are 3.0625, 0.5625, 0.0625,
# 5.0625, 1.5625, 1.5625; their sum is 11.875, so the population variance is
# 11.875 / 6 = 95/48 (the sample variance would be 11.875 / 5 = 2.375); at
# nr = 2 dB the scale is (95/48) / 10^0.2.
# ---------------------------------------------------------------------------
def test_noise_lambda_hand_worked_cube():
    tau_g = np.array([[0.0, 1.0, 2.0], [4.0, 0.5, 3.0]])
    p = _params(noise_mode="peak", peak_photons=100.0, dark_per_bin=1e-3)
    lam, scale, dark = oracle.noise_lambda(tau_g, p)
    assert scale == 25.0
    assert dark == float(np.float32(1e-3))
    want = np.array([[0.001, 25.001, 50.001], [100.001, 12.501, 75.001]], dtype=np.float32)
    np.testing.assert_allclose(lam, want, rtol=2e-7, atol=0)
    assert lam.dtype == np.float32 and lam.shape == (2, 3)

    p = _params(noise_mode="paper_nr", nr_db=2.0, dark_per_bin=0.0)
    lam, scale, dark = oracle.noise_lambda(tau_g, p)
    sigma_n = 1.9791666666666667 / 1.5848931924611136  # (95/48) / 10^(2/10)
    assert abs(scale - sigma_n) <= 1e-7 * sigma_n
    assert dark == 0.0
    np.testing.assert_allclose(lam, np.float32(sigma_n) * tau_g.astype(np.float32), rtol=2e-7)
    # a louder setting (larger nr) gives a smaller scale: fewer counts, more noise
    _, scale4, _ = oracle.noise_lambda(tau_g, dict(p, nr_db=4.0))
    assert abs(scale4 - 1.9791666666666667 / 2.51188643150958) <= 1e-7 * scale4
    # dark counts add to lambda in the paper mode as well
    lam_d, _, dark_d = oracle.noise_lambda(tau_g, dict(p, dark_per_bin=0.25))
    assert dark_d == 0.25
    np.testing.assert_allclose(lam_d, lam + np.float32(0.25), rtol=2e-7)


def test_noise_lambda_zero_cube():
    """An empty (all-zero) cube: no scale (no division by a zero peak)."""
    tau_g = np.zeros((3, 4))
    lam, scale, dark = oracle.noise_lambda(tau_g, _params(noise_mode="peak", dark_per_bin=1e-3))
    assert scale == 0.0
    np.testing.assert_array_equal(lam, np.full((3, 4), np.float32(1e-3)))
    lam, scale, _ = oracle.noise_lambda(tau_g, _params(noise_mode="paper_nr", dark_per_bin=0.0))
    assert scale == 0.0 and not lam.any()


# ---------------------------------------------------------------------------
# Splat forward: a single pair spreads w * N(b + 1/2 - u; 0, sigma) over the
# bins within 6 sigma (scipy's normal pdf), and the gradient matches central
# finite differences of the FP64 forward.
# ---------------------------------------------------------------------------
def test_splat_single_point_is_gaussian():
    stats = pytest.importorskip("scipy.stats")
    p = _params(scan_nx=1, scan_ny=1, wall_half_x=0.05, wall_half_y=0.05, bin_width_s=8e-12,
                num_bins=512, jitter_fwhm_s=60e-12, bin_mode="splat")
    pt = scenes.single_point(0.0, 0.0, 0.45, albedo=0.9, area=1e-3)  # u ~ 375
    u, w = oracle.pair(p, 0, pt[0])
    tau = oracle.forward_splat(p, pt)[0]
    sg = oracle.sigma_bins(60e-12, 8e-12)
    x = np.arange(512) + 0.5 - u
    ref = np.where(np.abs(x) < 6 * sg, w * stats.norm.pdf(x, scale=sg), 0.0)
    np.testing.assert_allclose(tau, ref, rtol=1e-13, atol=1e-300)
    assert tau.sum() == pytest.approx(w, rel=1e-8)


@pytest.mark.parametrize("scan_mode,cos_mode", [("confocal", "object"), ("confocal", "none"),
                                                ("nonconfocal", "object"),
                                                ("nonconfocal", "object_wall")])
def test_gradient_matches_central_differences(scan_mode, cos_mode):
    rng = np.random.default_rng(21)
    pts = scenes.random_points(rng, 12, half=0.3, z_lo=0.3, z_hi=0.5).astype(np.float64)
    p = _params(scan_nx=5, scan_ny=5, wall_half_x=0.4, wall_half_y=0.4, bin_width_s=8e-12,
                num_bins=400, jitter_fwhm_s=60e-12, bin_mode="splat", scan_mode=scan_mode,
                laser_xy=(0.05, -0.1), cos_mode=cos_mode, standoff_m=0.2,
                standoff_mode="euclidean")
    target = oracle.forward_splat(p, pts) * 0.9 + 1e-3 * rng.random((25, 400))

    def loss(pp):
        t = oracle.forward_splat(p, pp)
        return ((t - target) ** 2).sum()

    g = 2 * (oracle.forward_splat(p, pts) - target)
    ga, gd = oracle.backward_splat(p, pts, g)
    assert np.abs(gd).max() > 0 and np.abs(ga).max() > 0
    for i in range(pts.shape[0]):
        h = 1e-4  # the loss is quadratic in albedo: exact up to rounding
        a = pts.copy(); a[i, 6] += h
        b = pts.copy(); b[i, 6] -= h
        fd_a = (loss(a) - loss(b)) / (2 * h)
        assert ga[i] == pytest.approx(fd_a, rel=1e-6, abs=1e-9 * np.abs(ga).max())
        # depth: central differences converge as h^2; at h = 1e-6 m the truncation
        # error is ~1e-9 relative, at the workload's h = 1e-4 m it is ~1e-3
        for h, rel in [(1e-6, 1e-6), (1e-4, 5e-3)]:
            a = pts.copy(); a[i, 0:3] += h * pts[i, 3:6]
            b = pts.copy(); b[i, 0:3] -= h * pts[i, 3:6]
            fd_d = (loss(a) - loss(b)) / (2 * h)
            assert gd[i] == pytest.approx(fd_d, rel=rel, abs=1e-7 * np.abs(gd).max())
