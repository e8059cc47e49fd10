"""Seeded synthetic scenes for the NLOS transient simulator.

This module only builds INPUTS: hidden-surface samples and the scene/system
parameters. It holds none of the simulator's arithmetic (no path lengths, no
binning, no weights), so both the CUDA library and the CPU oracle can take
their inputs from it.

Inputs stand in for the paper's ShapeNet-derived depth maps (Simulation
section: 128x128 depth maps, 2 m x 2 m scan, 1024 bins, 32 ps), which are not
available here. Every generator is deterministic given its seed (numpy PCG64).

Point record (float32, 8 per point): x, y, z, nx, ny, nz, albedo, area, in
metres; the normal is a unit vector pointing away from the surface; the wall is
the plane z = 0 and hidden points have z > 0.

Parameters are a plain dict with the keys of ``default_params()``; times are in
seconds and lengths in metres.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 0x4E4C4F53  # workload k uses SEED_BASE + k


def default_params(**kw) -> dict:
    """Scene and system parameters (the paper's parameter list: relay surface
    extent and sampling, stand-off, bin width, window, jitter, noise)."""
    p = dict(
        scan_nx=32, scan_ny=32,
        wall_half_x=0.5, wall_half_y=0.5,
        scan_mode="confocal",          # or "nonconfocal"
        laser_xy=(0.0, 0.0),           # fixed laser spot (non-confocal)
        standoff_m=0.0,                # with "constant" and 0: no device legs (Eq. 1)
        standoff_mode="constant",      # "constant": 2*standoff; "euclidean": |D-l|+|d-D|
        bin_width_s=16e-12,
        num_bins=256,
        window_start_m=float("nan"),   # NaN: device legs of the wall centre
        jitter_fwhm_s=0.0,
        jitter_padding="zero",         # or "replicate" (the edge bins continue outside)
        bin_mode="nearest",            # or "splat"
        cos_mode="object",             # "none", "object", "object_wall"
        noise_mode="none",             # "none", "peak", "paper_nr"
        peak_photons=100.0,
        dark_per_bin=1e-3,
        nr_db=2.0,
        seed=0,
        stream_tag=0,
    )
    for k, v in kw.items():
        if k not in p:
            raise KeyError(f"unknown parameter {k!r}")
        p[k] = v
    return p


def _pack(xyz, nrm, albedo, area) -> np.ndarray:
    n = xyz.shape[0]
    out = np.empty((n, 8), dtype=np.float32)
    out[:, 0:3] = xyz
    out[:, 3:6] = nrm
    out[:, 6] = albedo
    out[:, 7] = area
    return out


def plane_grid(n: int, half: float, z: float, albedo, normal=(0.0, 0.0, -1.0)) -> np.ndarray:
    """n x n cell-centred samples of the square [-half, half]^2 at depth z,
    facing the wall; ``albedo`` is a scalar or an (n, n) array [iy, ix]."""
    c = -half + (np.arange(n) + 0.5) * (2.0 * half / n)
    X, Y = np.meshgrid(c, c)  # [iy, ix]
    xyz = np.stack([X.ravel(), Y.ravel(), np.full(n * n, z)], axis=1)
    nrm = np.tile(np.asarray(normal, dtype=np.float64), (n * n, 1))
    alb = np.broadcast_to(np.asarray(albedo, dtype=np.float64), (n, n)).ravel()
    area = np.full(n * n, (2.0 * half / n) ** 2)
    return _pack(xyz, nrm, alb, area)


def glyph(rng: np.random.Generator, blocks: int, upsample: int) -> np.ndarray:
    """A blocky binary albedo mask: blocks x blocks Bernoulli(0.5), upsampled."""
    g = (rng.random((blocks, blocks)) < 0.5).astype(np.float64)
    return np.kron(g, np.ones((upsample, upsample)))


# ---------------------------------------------------------------------------
# Workload 1: confocal 32x32 scan of a 1 m x 1 m wall, glyph plane at 0.5 m.
# ---------------------------------------------------------------------------
def workload_plane32(seed: int = SEED_BASE + 1):
    rng = np.random.default_rng(seed)
    params = default_params(scan_nx=32, scan_ny=32, wall_half_x=0.5, wall_half_y=0.5,
                            bin_width_s=16e-12, num_bins=256, standoff_m=0.0,
                            standoff_mode="constant", jitter_fwhm_s=0.0, noise_mode="none", seed=seed)
    pts = plane_grid(32, 0.5, 0.5, glyph(rng, 8, 4))
    return params, pts


# ---------------------------------------------------------------------------
# Workload 2: confocal 64x64 scan over 2 m x 2 m, 512 bins of 8 ps, stand-off
# 1 m; 262,144 area-uniform samples of a union of 3-6 spheres and boxes.
# ---------------------------------------------------------------------------
def _prim_union(rng):
    prims = []
    for _ in range(int(rng.integers(3, 7))):
        if rng.random() < 0.5:
            r = rng.uniform(0.1, 0.3)
            c = np.array([rng.uniform(-1 + r, 1 - r), rng.uniform(-1 + r, 1 - r),
                          rng.uniform(0.3 + r, 1.2 - r)])
            prims.append(("sphere", c, r))
        else:
            s = rng.uniform(0.1, 0.5, size=3)
            lo = np.array([rng.uniform(-1, 1 - s[0]), rng.uniform(-1, 1 - s[1]),
                           rng.uniform(0.3, 1.2 - s[2])])
            prims.append(("box", lo, lo + s))
    return prims


def _prim_area(pr):
    if pr[0] == "sphere":
        return 4.0 * math.pi * pr[2] ** 2
    s = pr[2] - pr[1]
    return 2.0 * (s[0] * s[1] + s[1] * s[2] + s[0] * s[2])


def _prim_sample(pr, rng, n):
    if pr[0] == "sphere":
        v = rng.normal(size=(n, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        return pr[1] + pr[2] * v, v
    lo, hi = pr[1], pr[2]
    s = hi - lo
    fa = np.array([s[1] * s[2], s[1] * s[2], s[0] * s[2], s[0] * s[2], s[0] * s[1], s[0] * s[1]])
    face = rng.choice(6, size=n, p=fa / fa.sum())
    p = lo + rng.random((n, 3)) * s
    nrm = np.zeros((n, 3))
    axis = face // 2
    side = face % 2
    idx = np.arange(n)
    p[idx, axis] = np.where(side == 0, lo[axis], hi[axis])
    nrm[idx, axis] = np.where(side == 0, -1.0, 1.0)
    return p, nrm


def _inside(pr, p):
    if pr[0] == "sphere":
        return np.linalg.norm(p - pr[1], axis=1) < pr[2]
    return np.all((p > pr[1]) & (p < pr[2]), axis=1)


def primitive_union_points(rng, n_points: int):
    prims = _prim_union(rng)
    areas = np.array([_prim_area(p) for p in prims])
    got_p, got_n = [], []
    n_acc = 0
    n_tried = 0
    while n_acc < n_points:
        m = max(4096, 2 * (n_points - n_acc))
        which = rng.choice(len(prims), size=m, p=areas / areas.sum())
        pos = np.empty((m, 3))
        nrm = np.empty((m, 3))
        for i, pr in enumerate(prims):
            sel = which == i
            pos[sel], nrm[sel] = _prim_sample(pr, rng, int(sel.sum()))
        keep = np.ones(m, dtype=bool)
        for i, pr in enumerate(prims):
            keep &= ~((which != i) & _inside(pr, pos))
        # count candidates up to (and including) the last one needed
        acc_idx = np.flatnonzero(keep)
        need = n_points - n_acc
        if acc_idx.size >= need:
            n_tried += int(acc_idx[need - 1]) + 1
            acc_idx = acc_idx[:need]
        else:
            n_tried += m
        got_p.append(pos[acc_idx])
        got_n.append(nrm[acc_idx])
        n_acc += acc_idx.size
    pos = np.concatenate(got_p)
    nrm = np.concatenate(got_n)
    acceptance = n_points / n_tried
    area = areas.sum() * acceptance / n_points
    albedo = rng.uniform(0.2, 1.0, size=n_points)
    return _pack(pos, nrm, albedo, np.full(n_points, area)), prims


def occluder_records(prims) -> np.ndarray:
    """The primitives of a union as occluder records [n, 8] (float32): kind 0
    sphere (centre, radius), kind 1 box (lower corner, upper corner)."""
    out = np.zeros((len(prims), 8), dtype=np.float32)
    for i, pr in enumerate(prims):
        if pr[0] == "sphere":
            out[i, 0] = 0
            out[i, 1:4] = pr[1]
            out[i, 4] = pr[2]
        else:
            out[i, 0] = 1
            out[i, 1:4] = pr[1]
            out[i, 4:7] = pr[2]
    return out


def workload_union64(seed: int = SEED_BASE + 2, n_points: int = 262144):
    """The acquisition window starts at the earliest object round trip seen
    from the wall centre (2 * stand-off + 2 * 0.3 m), so that it covers the
    nearest part of the scene."""
    rng = np.random.default_rng(seed)
    params = default_params(scan_nx=64, scan_ny=64, wall_half_x=1.0, wall_half_y=1.0,
                            bin_width_s=8e-12, num_bins=512, standoff_m=1.0,
                            standoff_mode="euclidean", window_start_m=2.0 * 1.0 + 2.0 * 0.3,
                            jitter_fwhm_s=60e-12,
                            noise_mode="peak", peak_photons=100.0, dark_per_bin=1e-3,
                            seed=seed)
    pts, _ = primitive_union_points(rng, n_points)
    return params, pts


# ---------------------------------------------------------------------------
# Workload 3: non-confocal (laser at the wall centre) 128x128 detector scan over
# 2 m x 2 m, 1024 bins of 4 ps, stand-off 1.5 m; 1024x1024 heightfield samples.
# ---------------------------------------------------------------------------
def heightfield_points(rng, n: int, half: float = 1.0, z_lo: float = 0.4, z_hi: float = 1.5,
                       n_bumps: int = 32):
    h = 2.0 * half / n
    c = -half + (np.arange(n) + 0.5) * h
    X, Y = np.meshgrid(c, c)  # [iy, ix]
    Z = np.zeros_like(X)
    for _ in range(n_bumps):
        cx, cy = rng.uniform(-half, half, size=2)
        sg = rng.uniform(0.1, 0.5)
        amp = rng.uniform(-1.0, 1.0)
        Z += amp * np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2.0 * sg * sg))
    Z = (Z - Z.min()) / (Z.max() - Z.min())
    Z = z_lo + (z_hi - z_lo) * Z
    dZdy, dZdx = np.gradient(Z, h, h)  # central differences inside, one-sided at the rim
    g2 = dZdx ** 2 + dZdy ** 2
    s = np.sqrt(1.0 + g2)
    nrm = np.stack([dZdx / s, dZdy / s, -1.0 / s], axis=-1).reshape(-1, 3)
    xyz = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    area = (h * h) * s.ravel()
    albedo = rng.beta(2.0, 2.0, size=n * n)
    return _pack(xyz, nrm, albedo, area)


def workload_heightfield128(seed: int = SEED_BASE + 3, n_side: int = 1024):
    """Window from the earliest round trip at the wall centre (2 * 1.5 + 2 * 0.4 m)."""
    rng = np.random.default_rng(seed)
    params = default_params(scan_nx=128, scan_ny=128, wall_half_x=1.0, wall_half_y=1.0,
                            scan_mode="nonconfocal", laser_xy=(0.0, 0.0),
                            bin_width_s=4e-12, num_bins=1024, standoff_m=1.5,
                            standoff_mode="euclidean", window_start_m=2.0 * 1.5 + 2.0 * 0.4,
                            jitter_fwhm_s=30e-12,
                            noise_mode="peak", peak_photons=100.0, dark_per_bin=1e-3,
                            seed=seed)
    pts = heightfield_points(rng, n_side)
    return params, pts


# ---------------------------------------------------------------------------
# Workload 4: batch of 8 confocal glyph-plane scenes (64x64 scan, 512 bins of
# 8 ps, 256x256 = 65,536 samples each, splat mode with 60 ps FWHM) and a target
# made from seeded depth (N(0, 2 mm) along the normal) and albedo (x U[0.8, 1.2])
# perturbations of the same scenes.
# ---------------------------------------------------------------------------
def workload_glyph_batch(seed: int = SEED_BASE + 4, n_scenes: int = 8, n_side: int = 256):
    rng = np.random.default_rng(seed)
    params = default_params(scan_nx=64, scan_ny=64, wall_half_x=0.5, wall_half_y=0.5,
                            bin_width_s=8e-12, num_bins=512, standoff_m=0.0,
                            jitter_fwhm_s=60e-12, bin_mode="splat", noise_mode="none",
                            seed=seed)
    scenes, targets = [], []
    for _ in range(n_scenes):
        z = rng.uniform(0.45, 0.55)
        pts = plane_grid(n_side, 0.5, z, glyph(rng, 8, n_side // 8))
        tgt = pts.copy()
        delta = rng.normal(0.0, 2e-3, size=pts.shape[0])
        tgt[:, 0:3] = pts[:, 0:3] + delta[:, None] * pts[:, 3:6]
        tgt[:, 6] = pts[:, 6] * rng.uniform(0.8, 1.2, size=pts.shape[0])
        scenes.append(pts)
        targets.append(tgt.astype(np.float32))
    return params, scenes, targets


# ---------------------------------------------------------------------------
# Workload 5: serving trace. Poisson arrivals; per request a log-uniform scan
# side in [16, 256], bins in [256, 2048], bin width in [4, 16] ps and point count
# in [1e4, 2e6]; confocal or non-confocal with probability 1/2; the scene comes
# from the union or the heightfield generator (coin flip).
# ---------------------------------------------------------------------------
def _log_uniform(rng, lo, hi):
    return math.exp(rng.uniform(math.log(lo), math.log(hi)))


def serving_trace(n_requests: int = 2000, rate_hz: float = 200.0, seed: int = SEED_BASE + 5,
                  side_range=(16, 256), bins_range=(256, 2048), dt_range=(4e-12, 16e-12),
                  points_range=(1e4, 2e6)):
    """Request descriptors (no points): arrival time, params, scene kind and seed."""
    rng = np.random.default_rng(seed)
    t = 0.0
    reqs = []
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        side = int(round(_log_uniform(rng, *side_range)))
        bins = int(round(_log_uniform(rng, *bins_range)))
        dt = _log_uniform(rng, *dt_range)
        npts = int(round(_log_uniform(rng, *points_range)))
        confocal = rng.random() < 0.5
        kind = "union" if rng.random() < 0.5 else "heightfield"
        fwhm = rng.uniform(30e-12, 70e-12)
        params = default_params(scan_nx=side, scan_ny=side, wall_half_x=1.0, wall_half_y=1.0,
                                scan_mode="confocal" if confocal else "nonconfocal",
                                bin_width_s=dt, num_bins=bins, standoff_m=1.0,
                                standoff_mode="euclidean",
                                window_start_m=2.0 + 2.0 * (0.3 if kind == "union" else 0.4),
                                jitter_fwhm_s=fwhm, noise_mode="peak", peak_photons=100.0,
                                dark_per_bin=1e-3, seed=rid)
        reqs.append(dict(id=rid, arrival_s=t, params=params, kind=kind, n_points=npts,
                         scene_seed=seed * 1000003 + rid))
    return reqs


def request_points(req) -> np.ndarray:
    """Surface samples of one serving request (generated on demand)."""
    rng = np.random.default_rng(req["scene_seed"])
    n = req["n_points"]
    if req["kind"] == "union":
        pts, _ = primitive_union_points(rng, n)
        return pts
    side = max(1, int(math.isqrt(n)))
    pts = heightfield_points(rng, side)
    return pts


def single_point(x, y, z, normal=(0.0, 0.0, -1.0), albedo=1.0, area=1.0) -> np.ndarray:
    return _pack(np.array([[x, y, z]]), np.array([normal]), np.array([albedo]), np.array([area]))


def random_points(rng, n, half=0.6, z_lo=0.2, z_hi=0.9) -> np.ndarray:
    """Uniform random samples with random normals roughly facing the wall."""
    xyz = np.stack([rng.uniform(-half, half, n), rng.uniform(-half, half, n),
                    rng.uniform(z_lo, z_hi, n)], axis=1)
    v = rng.normal(size=(n, 3))
    v[:, 2] = -np.abs(v[:, 2]) - 0.3
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return _pack(xyz, v, rng.uniform(0.1, 1.0, n), rng.uniform(1e-4, 4e-3, n))
