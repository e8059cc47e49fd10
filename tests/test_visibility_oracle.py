"""Pins of the oracle's visibility extension (occluders), against
formulations that share none of its code: dense sampling of a segment,
closed-form shadows of a sphere and of a box plate seen from one spot, the
laser leg of a non-confocal scan, and brute-force sampled visibility on a
small union of primitives.

The paper's model (Eq. 1) has no visibility term; the occluder reading is:
a pair is dropped when a segment from one of its spots to the point runs
inside an occluder (sphere or axis-aligned box) for more than a fraction eta
of its length.
"""
import numpy as np
import pytest

import oracle
import scenes

ETA = oracle.OCC_ETA


def _inside(rec, P):
    """Strictly inside the occluder (plain definition), P [..., 3]."""
    kind = int(rec[0])
    a = np.asarray(rec[1:4], dtype=np.float64)
    b = np.asarray(rec[4:7], dtype=np.float64)
    if kind == 0:
        return np.sum((P - a) ** 2, axis=-1) < b[0] ** 2
    return np.all((P > a) & (P < b), axis=-1)


def _sampled_chord(rec, x, y, n=200000):
    t = (np.arange(n) + 0.5) / n
    P = np.asarray(x, np.float64)[None, :] + t[:, None] * (np.asarray(y, np.float64) - x)[None, :]
    return _inside(rec, P).mean()


def _f32(v):
    return np.asarray(v, dtype=np.float32).astype(np.float64)


def test_chord_matches_dense_sampling():
    rng = np.random.default_rng(11)
    n = 200000
    cases = 0
    for i in range(60):
        if rng.random() < 0.5:
            cen = rng.uniform(-0.5, 0.5, 3)
            rec = _f32([0, *cen, rng.uniform(0.1, 0.6), 0, 0, 0])
        else:
            lo = rng.uniform(-0.6, 0.2, 3)
            hi = lo + rng.uniform(0.1, 0.7, 3)
            cen = 0.5 * (lo + hi)
            rec = _f32([1, *lo, *hi, 0])
        x = rng.uniform(-1, 1, 3)
        # every other segment is aimed near the solid, so that many cross it
        y = cen + rng.uniform(-0.3, 0.3, 3) if i % 2 else rng.uniform(-1, 1, 3)
        c = oracle.chord(rec, x, y)
        est = _sampled_chord(rec, x, y, n)
        assert abs(c - est) <= 3.0 / n, (rec, x, y, c, est)
        cases += c > 0
    assert cases >= 10  # the draw exercises intersecting segments
    # segments along a box face, through a corner region, starting and ending inside
    box = _f32([1, -0.5, -0.5, -0.5, 0.5, 0.5, 0.5, 0])
    assert oracle.chord(box, [-1, 0.5, 0], [1, 0.5, 0]) == 0.0  # on the face plane: not inside
    assert oracle.chord(box, [-1, 0.2, 0], [1, 0.2, 0]) == pytest.approx(0.5, abs=1e-15)
    assert oracle.chord(box, [0, 0, 0], [0, 0, 2]) == pytest.approx(0.25, abs=1e-15)
    assert oracle.chord(box, [0, 0, 0], [0.1, 0.1, 0.1]) == pytest.approx(1.0, abs=1e-15)
    sph = _f32([0, 0, 0, 0, 0.5, 0, 0, 0])
    assert oracle.chord(sph, [0, 0.5, -1], [0, 0.5, 1]) == 0.0  # tangent line
    assert oracle.chord(sph, [0, 0, 0], [0, 0, 2]) == pytest.approx(0.25, abs=1e-15)


def _spot_params(**kw):
    # one scan point at the origin of the wall, no stand-off, a long window
    p = scenes.default_params(scan_nx=1, scan_ny=1, wall_half_x=0.5, wall_half_y=0.5,
                              bin_width_s=16e-12, num_bins=1024, standoff_m=0.0,
                              standoff_mode="constant", cos_mode="object")
    p.update(kw)
    return p


def test_far_occluder_changes_nothing():
    params, pts = scenes.workload_plane32()
    far = [[0, 0.0, 0.0, -5.0, 0.5, 0, 0, 0], [1, 3.0, 3.0, 0.2, 4.0, 4.0, 2.0, 0]]
    plain = oracle.forward_binned(params, pts)["tau"]
    vis = oracle.forward_binned(params, pts, occ=far)
    assert np.array_equal(plain, vis["tau"])
    assert vis["n_occ_border"] == 0


def test_sphere_shadow_closed_form():
    """Spot at the origin, plane of points at z0 = 1, sphere of radius r centred
    on the axis at depth zc: the line from the origin towards X passes the
    centre at distance h = |c x X| / |X|, and its chord is 2 sqrt(r^2 - h^2),
    i.e. 2 sqrt(r^2 - h^2) / |X| of the segment."""
    params = _spot_params()
    pts = scenes.plane_grid(64, 0.5, 1.0, 1.0)
    zc, r = 0.5, 0.1
    occ = [[0, 0.0, 0.0, zc, r, 0, 0, 0]]
    X = pts[:, :3].astype(np.float64)
    c = np.array([0.0, 0.0, zc])
    h2 = np.sum(np.cross(c[None, :], X) ** 2, axis=1) / np.sum(X ** 2, axis=1)
    chord = np.where(h2 < r * r, 2.0 * np.sqrt(np.maximum(r * r - h2, 0.0)), 0.0) / np.linalg.norm(X, axis=1)
    assert np.min(np.abs(chord - ETA)) > 1e-6  # no point sits on the threshold
    hidden = chord > ETA
    assert 30 < hidden.sum() < len(pts) - 30
    got = oracle.forward_binned(params, pts, occ=occ)["tau"]
    want = oracle.forward_binned(params, pts[~hidden])["tau"]
    assert np.array_equal(got, want)


def test_box_plate_closed_form():
    """A plate lo < (x, y, z) < hi between the spot (origin) and the plane z0 = 1:
    the ray towards X = (x, y, 1) is at (x z, y z) at depth z, so its chord is
    the measure of the depths z in (lo_z, hi_z) with lo_x < x z < hi_x and
    lo_y < y z < hi_y (each an interval of z), divided by |X| / |X| = z0 = 1."""
    params = _spot_params()
    pts = scenes.plane_grid(80, 0.5, 1.0, 1.0)
    lo = np.array([-0.17, -0.11, 0.40])
    hi = np.array([0.23, 0.19, 0.46])
    occ = [[1, *lo, *hi, 0]]
    lo32, hi32 = _f32(lo), _f32(hi)
    X = pts[:, :3].astype(np.float64)
    zlo = np.full(len(X), lo32[2])
    zhi = np.full(len(X), hi32[2])
    for k in range(2):
        v = X[:, k] / X[:, 2]  # lateral position per unit depth
        with np.errstate(divide="ignore"):
            a = np.where(v > 0, lo32[k] / v, np.where(v < 0, hi32[k] / v, -np.inf))
            b = np.where(v > 0, hi32[k] / v, np.where(v < 0, lo32[k] / v, np.inf))
        zero_ok = (lo32[k] < 0) & (0 < hi32[k])
        a = np.where(v == 0, np.where(zero_ok, -np.inf, np.inf), a)
        b = np.where(v == 0, np.where(zero_ok, np.inf, -np.inf), b)
        zlo = np.maximum(zlo, a)
        zhi = np.minimum(zhi, b)
    chord = np.maximum(zhi - zlo, 0.0) / X[:, 2]  # segment from depth 0 to depth z0
    assert np.min(np.abs(chord - ETA)) > 1e-7
    hidden = chord > ETA
    assert 30 < hidden.sum() < len(pts) - 30
    got = oracle.forward_binned(params, pts, occ=occ)["tau"]
    want = oracle.forward_binned(params, pts[~hidden])["tau"]
    assert np.array_equal(got, want)


def test_nonconfocal_laser_leg():
    """Non-confocal: a point hidden from the laser spot is dark for every
    detector spot; a point hidden only from some detector spots is missing
    from those transients alone. Visibility from each spot by the sphere's
    closed form (distance of the centre from the segment's line)."""
    params = scenes.default_params(scan_nx=4, scan_ny=4, wall_half_x=0.5, wall_half_y=0.5,
                                   scan_mode="nonconfocal", laser_xy=(0.45, 0.0),
                                   bin_width_s=16e-12, num_bins=1024, standoff_m=0.0,
                                   standoff_mode="constant", cos_mode="object")
    pts = scenes.plane_grid(24, 0.4, 0.9, 1.0)
    cen = np.array([0.3, 0.05, 0.45])
    r = 0.08
    occ = [[0, *cen, r, 0, 0, 0]]
    c32 = _f32(cen)
    r32 = float(np.float32(r))
    X = pts[:, :3].astype(np.float64)

    def hidden_from(z):
        d = X - z
        f = z - c32
        A = np.sum(d * d, axis=1)
        Bq = np.sum(f * d, axis=1)
        h2 = np.sum(f * f) - Bq * Bq / A  # squared distance of the centre from the line
        half = np.sqrt(np.maximum(r32 * r32 - h2, 0.0)) / np.sqrt(A)
        mid = -Bq / A
        chord = np.clip(np.minimum(mid + half, 1.0) - np.maximum(mid - half, 0.0), 0.0, None)
        chord = np.where(h2 < r32 * r32, chord, 0.0)
        assert np.min(np.abs(chord - ETA)) > 1e-7
        return chord > ETA

    laser = np.array([params["laser_xy"][0], params["laser_xy"][1], 0.0])
    hid_l = hidden_from(laser)
    assert 5 < hid_l.sum() < len(pts) - 5
    got = oracle.forward_binned(params, pts, occ=occ)["tau"]
    for s in range(16):
        spot = np.array(oracle.scan_geometry(params, s)[1])
        keep = ~(hid_l | hidden_from(spot))
        want = oracle.forward_binned(params, pts[keep], s_begin=s, s_count=1)["tau"][0]
        assert np.array_equal(got[s], want), s


@pytest.mark.parametrize("cos_mode", ["object", "none"])
def test_union_self_occlusion_sampled(cos_mode):
    """Primitive union with its own primitives as occluders: per (spot, point),
    visibility from a 4000-sample chord estimate; pairs the estimate cannot
    decide (within 3 samples of the threshold) are compared through their
    weight as an allowance."""
    rng = np.random.default_rng(scenes.SEED_BASE + 2)
    pts, prims = scenes.primitive_union_points(rng, 400)
    occ = []
    for pr in prims:
        if pr[0] == "sphere":
            occ.append([0, *pr[1], pr[2], 0, 0, 0])
        else:
            occ.append([1, *pr[1], *pr[2], 0])
    occ32 = np.asarray(occ, dtype=np.float32).astype(np.float64)
    params = scenes.default_params(scan_nx=3, scan_ny=3, wall_half_x=1.0, wall_half_y=1.0,
                                   bin_width_s=16e-12, num_bins=1024, standoff_m=0.0,
                                   standoff_mode="constant", cos_mode=cos_mode)
    n = 4000
    t = (np.arange(n) + 0.5) / n
    X = pts[:, :3].astype(np.float64)
    got = oracle.forward_binned(params, pts, occ=occ)["tau"]
    u, w = oracle.pair_table(params, pts, np.arange(9))
    n_hidden = 0
    for s in range(9):
        spot = np.array(oracle.scan_geometry(params, s)[1])
        seg = spot[None, None, :] + t[None, :, None] * (X - spot)[:, None, :]  # [P, n, 3]
        est = np.zeros((len(X), len(occ32)))
        for k, rec in enumerate(occ32):
            est[:, k] = _inside(rec, seg).mean(axis=1)
        hidden = (est > ETA).any(axis=1)
        unsure = (np.abs(est - ETA) <= 3.0 / n).any(axis=1)
        n_hidden += int((hidden & (w[s] != 0)).sum())
        want = np.zeros(1024)
        allow = np.zeros(1024)
        inw = (u[s] >= 0) & (u[s] < 1024)
        b = np.floor(u[s]).astype(np.int64)
        sel = inw & ~hidden & ~unsure
        np.add.at(want, b[sel], w[s][sel])
        np.add.at(allow, b[inw & unsure], np.abs(w[s][inw & unsure]))
        err = np.abs(got[s] - want)
        assert np.all(err <= allow + 1e-12 * np.abs(want).max() + 1e-300), s
    assert n_hidden > 0  # the scene does shadow itself


def test_threshold_one_hides_nothing_and_more_occluders_only_remove_light():
    """Invariants: a chord never exceeds the whole segment, so with eta = 1 no
    pair is hidden (the plain forward, bit for bit); and every pair hidden by a
    set of occluders stays hidden when occluders are added, so each bin can only
    lose weight."""
    rng = np.random.default_rng(scenes.SEED_BASE + 2)
    pts, prims = scenes.primitive_union_points(rng, 600)
    occ = scenes.occluder_records(prims)
    params = scenes.default_params(scan_nx=4, scan_ny=3, wall_half_x=1.0, wall_half_y=1.0,
                                   bin_width_s=16e-12, num_bins=1024, standoff_m=0.0,
                                   standoff_mode="constant", cos_mode="none")
    plain = oracle.forward_binned(params, pts)["tau"]
    assert np.array_equal(oracle.forward_binned(params, pts, occ=occ, eta=1.0)["tau"], plain)
    prev = plain
    for k in range(1, len(occ) + 1):
        cur = oracle.forward_binned(params, pts, occ=occ[:k])["tau"]
        assert np.all(cur <= prev + 1e-12 * plain.max())
        prev = cur
    assert prev.sum() < plain.sum()
