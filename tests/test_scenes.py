"""The seeded synthetic workloads against their stated recipes: sizes and
parameters, the geometry of the samples (on the primitives' surfaces, unit
outward normals, the heightfield's normals and areas from its own central
differences), the value distributions, and the serving trace's log-uniform
means in closed form. No simulator arithmetic is involved."""
import math

import numpy as np
import pytest

import scenes

C_PS = 1e-12


def _unit(n, tol=1e-6):
    return np.all(np.abs(np.linalg.norm(n.astype(np.float64), axis=1) - 1.0) < tol)


def test_generators_are_deterministic():
    a = scenes.workload_union64(n_points=5000)[1]
    b = scenes.workload_union64(n_points=5000)[1]
    assert np.array_equal(a, b)
    c = scenes.workload_union64(seed=scenes.SEED_BASE + 99, n_points=5000)[1]
    assert not np.array_equal(a, c)
    h1 = scenes.workload_heightfield128(n_side=64)[1]
    h2 = scenes.workload_heightfield128(n_side=64)[1]
    assert np.array_equal(h1, h2)


def test_plane32_recipe():
    p, pts = scenes.workload_plane32()
    assert (p["scan_nx"], p["scan_ny"], p["num_bins"]) == (32, 32, 256)
    assert p["bin_width_s"] == pytest.approx(16 * C_PS)
    assert (p["wall_half_x"], p["standoff_m"], p["jitter_fwhm_s"], p["noise_mode"]) == \
        (0.5, 0.0, 0.0, "none")
    assert pts.shape == (1024, 8) and pts.dtype == np.float32
    assert np.all(pts[:, 2] == np.float32(0.5))
    assert np.all(pts[:, 3:6] == np.array([0, 0, -1], dtype=np.float32))
    assert np.allclose(pts[:, 7], (1.0 / 32) ** 2)
    # cell-centred grid over [-0.5, 0.5]^2
    xs = np.unique(pts[:, 0])
    assert xs.size == 32 and np.allclose(xs, -0.5 + (np.arange(32) + 0.5) / 32)
    # the albedo is a binary glyph of 8 x 8 blocks, each 4 x 4 samples
    a = pts[:, 6].reshape(32, 32)
    assert set(np.unique(a)) <= {0.0, 1.0}
    blocks = a.reshape(8, 4, 8, 4)
    assert np.all(blocks == blocks[:, :1, :, :1])


def _on_surface(prims, pos, nrm):
    """For each sample: the distance to the surface of the primitive it lies
    on and the angle error of its normal against that surface's outward one."""
    best_d = np.full(pos.shape[0], np.inf)
    best_e = np.full(pos.shape[0], np.inf)
    for pr in prims:
        if pr[0] == "sphere":
            v = pos - pr[1]
            r = np.linalg.norm(v, axis=1)
            d = np.abs(r - pr[2])
            e = np.linalg.norm(nrm - v / r[:, None], axis=1)
        else:
            lo, hi = np.asarray(pr[1]), np.asarray(pr[2])
            inside = np.all((pos >= lo - 1e-6) & (pos <= hi + 1e-6), axis=1)
            dist_lo, dist_hi = np.abs(pos - lo), np.abs(pos - hi)
            face = np.minimum(dist_lo, dist_hi)
            axis = np.argmin(face, axis=1)
            d = np.where(inside, face[np.arange(pos.shape[0]), axis], np.inf)
            want = np.zeros_like(pos)
            sign = np.where(dist_lo[np.arange(pos.shape[0]), axis] <
                            dist_hi[np.arange(pos.shape[0]), axis], -1.0, 1.0)
            want[np.arange(pos.shape[0]), axis] = sign
            e = np.linalg.norm(nrm - want, axis=1)
        better = d < best_d
        best_d = np.where(better, d, best_d)
        best_e = np.where(better, e, best_e)
    return best_d, best_e


def test_union64_recipe():
    p, pts = scenes.workload_union64()
    assert (p["scan_nx"], p["scan_ny"], p["num_bins"], p["scan_mode"]) == (64, 64, 512, "confocal")
    assert p["bin_width_s"] == pytest.approx(8 * C_PS)
    assert (p["wall_half_x"], p["standoff_m"], p["standoff_mode"]) == (1.0, 1.0, "euclidean")
    assert p["window_start_m"] == pytest.approx(2.6)
    assert p["jitter_fwhm_s"] == pytest.approx(60 * C_PS)
    assert (p["noise_mode"], p["peak_photons"], p["dark_per_bin"]) == ("peak", 100.0, 1e-3)
    assert pts.shape == (262144, 8)
    assert np.all((pts[:, 2] >= 0.3 - 1e-6) & (pts[:, 2] <= 1.2 + 1e-6))
    assert np.all(np.abs(pts[:, 0:2]) <= 1.0 + 1e-6)
    assert np.all((pts[:, 6] >= 0.2) & (pts[:, 6] <= 1.0))
    assert np.unique(pts[:, 7]).size == 1 and pts[0, 7] > 0
    assert _unit(pts[:, 3:6])


def test_union_samples_lie_on_their_primitives():
    rng = np.random.default_rng(scenes.SEED_BASE + 2)
    pts, prims = scenes.primitive_union_points(rng, 20000)
    assert 3 <= len(prims) <= 6
    pos, nrm = pts[:, 0:3].astype(np.float64), pts[:, 3:6].astype(np.float64)
    d, e = _on_surface(prims, pos, nrm)
    assert d.max() < 1e-5 and e.max() < 1e-5
    # no sample strictly inside another primitive
    for pr in prims:
        if pr[0] == "sphere":
            inside = np.linalg.norm(pos - pr[1], axis=1) < pr[2] - 1e-5
        else:
            inside = np.all((pos > np.asarray(pr[1]) + 1e-5) & (pos < np.asarray(pr[2]) - 1e-5),
                            axis=1)
        assert not inside.any()
    # the patch area times the count is the union's visible area <= the sum of areas
    total = sum(4 * math.pi * pr[2] ** 2 if pr[0] == "sphere" else
                2 * float(np.prod(np.asarray(pr[2]) - pr[1]) *
                          np.sum(1.0 / (np.asarray(pr[2]) - pr[1]))) for pr in prims)
    assert 0 < pts[0, 7] * pts.shape[0] <= total * (1 + 1e-6)


def test_heightfield128_recipe():
    p, pts = scenes.workload_heightfield128()
    assert (p["scan_nx"], p["scan_ny"], p["num_bins"], p["scan_mode"]) == \
        (128, 128, 1024, "nonconfocal")
    assert tuple(p["laser_xy"]) == (0.0, 0.0)
    assert p["bin_width_s"] == pytest.approx(4 * C_PS)
    assert (p["wall_half_x"], p["standoff_m"], p["standoff_mode"]) == (1.0, 1.5, "euclidean")
    assert p["window_start_m"] == pytest.approx(3.8)
    assert p["jitter_fwhm_s"] == pytest.approx(30 * C_PS)
    n = 1024
    h = 2.0 / n
    assert pts.shape == (n * n, 8)
    z = pts[:, 2].astype(np.float64)
    assert z.min() == pytest.approx(0.4, abs=1e-6) and z.max() == pytest.approx(1.5, abs=1e-6)
    nrm = pts[:, 3:6].astype(np.float64)
    assert _unit(nrm) and np.all(nrm[:, 2] < 0)
    # area = cell * sqrt(1 + |grad z|^2) = cell / |n_z|
    assert np.allclose(pts[:, 7], h * h / -nrm[:, 2], rtol=1e-5)
    # interior normals follow the central differences of the sampled heights
    Z = z.reshape(n, n)
    gx = (Z[1:-1, 2:] - Z[1:-1, :-2]) / (2 * h)
    gy = (Z[2:, 1:-1] - Z[:-2, 1:-1]) / (2 * h)
    s = np.sqrt(1 + gx ** 2 + gy ** 2)
    N = nrm.reshape(n, n, 3)[1:-1, 1:-1]
    assert np.allclose(N[..., 0], gx / s, atol=2e-4)
    assert np.allclose(N[..., 1], gy / s, atol=2e-4)
    # albedo Beta(2, 2): mean 1/2, variance 1/20
    a = pts[:, 6].astype(np.float64)
    assert np.all((a > 0) & (a < 1))
    assert a.mean() == pytest.approx(0.5, abs=3e-3)
    assert a.var() == pytest.approx(0.05, abs=1e-3)


def test_glyph_batch_recipe():
    p, sc, tg = scenes.workload_glyph_batch()
    assert (p["scan_nx"], p["num_bins"], p["bin_mode"], p["scan_mode"]) == (64, 512, "splat", "confocal")
    assert p["bin_width_s"] == pytest.approx(8 * C_PS) and p["jitter_fwhm_s"] == pytest.approx(60 * C_PS)
    assert len(sc) == len(tg) == 8
    deltas, ratios = [], []
    for pts, t in zip(sc, tg):
        assert pts.shape == (65536, 8)
        z0 = float(pts[0, 2])
        assert 0.45 <= z0 <= 0.55 and np.all(pts[:, 2] == pts[0, 2])
        a = pts[:, 6].reshape(256, 256)
        assert set(np.unique(a)) <= {0.0, 1.0}
        blocks = a.reshape(8, 32, 8, 32)
        assert np.all(blocks == blocks[:, :1, :, :1])
        # the target moves each point along its normal (0, 0, -1) and scales its albedo
        assert np.allclose(t[:, 0:2], pts[:, 0:2]) and np.array_equal(t[:, 3:6], pts[:, 3:6])
        deltas.append(pts[:, 2].astype(np.float64) - t[:, 2])
        lit = pts[:, 6] > 0
        ratios.append(t[lit, 6].astype(np.float64) / pts[lit, 6])
    d = np.concatenate(deltas)
    assert abs(d.mean()) < 5e-5 and d.std() == pytest.approx(2e-3, rel=0.02)
    r = np.concatenate(ratios)
    assert r.min() >= 0.8 - 1e-6 and r.max() <= 1.2 + 1e-6
    assert r.mean() == pytest.approx(1.0, abs=2e-3)


def test_serving_trace_recipe():
    reqs = scenes.serving_trace()
    assert len(reqs) == 2000
    t = np.array([r["arrival_s"] for r in reqs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0) and gaps.mean() == pytest.approx(1 / 200.0, rel=0.07)
    side = np.array([r["params"]["scan_nx"] for r in reqs], dtype=np.float64)
    bins = np.array([r["params"]["num_bins"] for r in reqs])
    dt = np.array([r["params"]["bin_width_s"] for r in reqs])
    P = np.array([r["n_points"] for r in reqs], dtype=np.float64)
    assert side.min() >= 16 and side.max() <= 256
    assert bins.min() >= 256 and bins.max() <= 2048
    assert dt.min() >= 4 * C_PS and dt.max() <= 16 * C_PS
    assert P.min() >= 1e4 and P.max() <= 2e6
    # log-uniform on [a, b]: E[x] = (b - a) / ln(b / a), E[x^2] = (b^2 - a^2) / (2 ln(b / a))
    assert P.mean() == pytest.approx((2e6 - 1e4) / math.log(200.0), rel=0.1)
    assert (side ** 2).mean() == pytest.approx((256 ** 2 - 16 ** 2) / (2 * math.log(16.0)), rel=0.1)
    conf = np.mean([r["params"]["scan_mode"] == "confocal" for r in reqs])
    union = np.mean([r["kind"] == "union" for r in reqs])
    assert abs(conf - 0.5) < 0.05 and abs(union - 0.5) < 0.05
    assert len({r["scene_seed"] for r in reqs}) == 2000
