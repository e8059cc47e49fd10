"""FP64 CPU oracle of the NLOS transient simulator (arXiv 2506.03747).

TEST INFRASTRUCTURE ONLY. The test suite, the smoke check and the benchmark's
CPU-baseline leg are its only users; the product path (the CUDA library and its
Python binding) never imports it, and the two share no code.

The arithmetic lives in ``nlos_oracle.c`` (plain C, double precision, brute
force over all pairs); this module compiles it with gcc on first use and
marshals numpy arrays. Inputs are the float32 point records of ``scenes``,
promoted exactly to float64.

Pinned by the ``-m "not gpu"`` tests against closed forms, invariants, a
50-digit brute force and the curand Philox generator; the FP32 Poisson
sampler is pinned statistically against the Poisson distribution.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nlos_oracle.c")
_LIB_PATH = os.path.join(_HERE, "libnlos_oracle.so")
_lock = threading.Lock()
_lib = None

LIGHT_SPEED = 299792458.0


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, OpenMP, no fast-math,
    no FP contraction so that results do not depend on the host ISA)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "nlos_oracle.h"))):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", "-fopenmp",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Geom(ctypes.Structure):
    _fields_ = [
        ("scan_nx", ctypes.c_int32), ("scan_ny", ctypes.c_int32),
        ("wall_half_x", ctypes.c_double), ("wall_half_y", ctypes.c_double),
        ("nonconfocal", ctypes.c_int32),
        ("laser_x", ctypes.c_double), ("laser_y", ctypes.c_double),
        ("standoff", ctypes.c_double), ("standoff_mode", ctypes.c_int32),
        ("bin_width_s", ctypes.c_double), ("num_bins", ctypes.c_int32),
        ("window_start_m", ctypes.c_double),
        ("cos_mode", ctypes.c_int32),
    ]


_COS = {"none": 0, "object": 1, "object_wall": 2}


def geom(params: dict) -> Geom:
    return Geom(
        scan_nx=int(params["scan_nx"]), scan_ny=int(params["scan_ny"]),
        wall_half_x=float(params["wall_half_x"]), wall_half_y=float(params["wall_half_y"]),
        nonconfocal=1 if params["scan_mode"] == "nonconfocal" else 0,
        laser_x=float(params["laser_xy"][0]), laser_y=float(params["laser_xy"][1]),
        standoff=float(params["standoff_m"]),
        standoff_mode=1 if params["standoff_mode"] == "constant" else 0,
        bin_width_s=float(params["bin_width_s"]), num_bins=int(params["num_bins"]),
        window_start_m=float(params["window_start_m"]),
        cos_mode=_COS[params["cos_mode"]],
    )


class Occluder(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("a", ctypes.c_double * 3), ("b", ctypes.c_double * 3)]


# Visibility threshold: a segment is blocked when its chord inside an occluder
# exceeds this fraction of its length (a reading of this build; the paper's
# model has no visibility term).
OCC_ETA = 4e-3


def occluders(recs) -> ctypes.Array:
    """Occluder records [n, 8] (kind, a0, a1, a2, b0, b1, b2, unused; kind 0 =
    sphere with centre a and radius b0, kind 1 = box with corners a < b), as
    float32 values promoted exactly to float64."""
    r = np.asarray(recs, dtype=np.float32).reshape(-1, 8).astype(np.float64)
    arr = (Occluder * max(1, len(r)))()
    for i, o in enumerate(r):
        arr[i].kind = int(o[0])
        for k in range(3):
            arr[i].a[k] = o[1 + k]
            arr[i].b[k] = o[4 + k]
    return arr


def chord(rec, x, y) -> float:
    """Fraction of segment x -> y strictly inside the occluder ``rec``."""
    lib = _load()
    o = occluders([rec])
    xa = np.ascontiguousarray(x, dtype=np.float64)
    ya = np.ascontiguousarray(y, dtype=np.float64)
    return float(lib.orc_chord(o, _ptr(xa), _ptr(ya)))


_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
_GP = ctypes.POINTER(Geom)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.orc_scan_geometry.argtypes = [_GP, _I64, _P, _P, _P]
            lib.orc_window_start.argtypes = [_GP]
            lib.orc_window_start.restype = _D
            lib.orc_pair.argtypes = [_GP, _I64, _P, _P, _P]
            lib.orc_pair_table.argtypes = [_GP, _I64, _P, _P, _I64, _P, _P, ctypes.c_int]
            lib.orc_forward_binned.argtypes = [_GP, _I64, _P, _I64, _I64, _P, _D, _P, _P, _P,
                                               ctypes.c_int]
            lib.orc_chord.argtypes = [ctypes.POINTER(Occluder), _P, _P]
            lib.orc_chord.restype = _D
            lib.orc_forward_binned_vis.argtypes = [_GP, _I64, _P, _I64, _I64,
                                                   ctypes.POINTER(Occluder), ctypes.c_int32, _D,
                                                   _D, _P, _D, _P, _P, _P, _P, _P, ctypes.c_int]
            lib.orc_jitter_taps.argtypes = [_D, _D, _P, ctypes.c_int]
            lib.orc_jitter.argtypes = [_P, _I64, ctypes.c_int32, _P, ctypes.c_int32, _P]
            lib.orc_jitter_padded.argtypes = [_P, _I64, ctypes.c_int32, _P, ctypes.c_int32,
                                              ctypes.c_int32, _P]
            lib.orc_philox4x32_10.argtypes = [_P, _P, _P]
            lib.orc_philox_many.argtypes = [_P, _I64, _P, _P]
            lib.orc_noise_lambda.argtypes = [_P, _I64, ctypes.c_float, ctypes.c_float, _P]
            lib.orc_poisson_one.argtypes = [ctypes.c_float, ctypes.c_uint64, ctypes.c_uint64,
                                            ctypes.c_uint32]
            lib.orc_poisson_one.restype = ctypes.c_uint32
            lib.orc_poisson.argtypes = [_P, _I64, ctypes.c_uint64, ctypes.c_uint64,
                                        ctypes.c_uint32, _P, ctypes.c_int]
            lib.orc_forward_splat.argtypes = [_GP, _D, _I64, _P, _I64, _I64, _P, ctypes.c_int]
            lib.orc_backward_splat.argtypes = [_GP, _D, _I64, _P, _P, _P, _P, ctypes.c_int]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _pts64(pts) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(pts), dtype=np.float64)
    if a.ndim != 2 or a.shape[1] != 8:
        raise ValueError("points must be [P, 8]")
    return a


def num_scan(params) -> int:
    return int(params["scan_nx"]) * int(params["scan_ny"])


def scan_geometry(params, s: int):
    lib = _load()
    g = geom(params)
    l = np.zeros(3)
    d = np.zeros(3)
    legs = np.zeros(1)
    lib.orc_scan_geometry(ctypes.byref(g), int(s), _ptr(l), _ptr(d), _ptr(legs))
    return l, d, float(legs[0])


def window_start(params) -> float:
    g = geom(params)
    return float(_load().orc_window_start(ctypes.byref(g)))


def pair(params, s: int, pt):
    lib = _load()
    g = geom(params)
    p = np.ascontiguousarray(np.asarray(pt, dtype=np.float64).reshape(8))
    u = np.zeros(1)
    w = np.zeros(1)
    lib.orc_pair(ctypes.byref(g), int(s), _ptr(p), _ptr(u), _ptr(w))
    return float(u[0]), float(w[0])


def pair_table(params, pts, scan_ids, threads: int = 0):
    """u[i, p], w[i, p] for the scan points in ``scan_ids``."""
    lib = _load()
    g = geom(params)
    P = _pts64(pts)
    ids = np.ascontiguousarray(np.asarray(scan_ids, dtype=np.int64))
    u = np.zeros((ids.size, P.shape[0]))
    w = np.zeros((ids.size, P.shape[0]))
    lib.orc_pair_table(ctypes.byref(g), P.shape[0], _ptr(P), _ptr(ids), ids.size, _ptr(u),
                       _ptr(w), threads)
    return u, w


def forward_binned(params, pts, s_begin: int = 0, s_count: int | None = None,
                   eps: float = 0.0, threads: int = 0, occ=None, eta: float = OCC_ETA,
                   occ_delta: float = 0.0):
    """Binned transient tau[s, b] (float64) for scan points s_begin..s_begin+s_count.

    With eps > 0 also returns the per-bin mass of pairs within eps of a bin edge
    (``flip_mass``), its window-edge part (``edge_mass``) and their count.
    With occluder records ``occ`` ([n, 8], see ``occluders``), pairs whose point
    is hidden from one of its spots are left out; ``occ_mass`` / ``n_occ_border``
    are the weight and count of pairs whose chord lies within ``occ_delta`` of
    ``eta``."""
    if occ is not None and len(np.asarray(occ).reshape(-1, 8)) > 0:
        return _forward_binned_vis(params, pts, s_begin, s_count, eps, threads, occ, eta,
                                   occ_delta)
    lib = _load()
    g = geom(params)
    P = _pts64(pts)
    S = num_scan(params)
    if s_count is None:
        s_count = S - s_begin
    if not (0 <= s_begin and s_begin + s_count <= S):
        raise ValueError("scan range out of bounds")
    B = int(params["num_bins"])
    tau = np.zeros((s_count, B))
    flip = np.zeros((s_count, B)) if eps > 0 else None
    edge = np.zeros(s_count) if eps > 0 else None
    nb = np.zeros(1, dtype=np.int64)
    lib.orc_forward_binned(ctypes.byref(g), P.shape[0], _ptr(P), s_begin, s_count, _ptr(tau),
                           float(eps), _ptr(flip) if flip is not None else None,
                           _ptr(edge) if edge is not None else None, _ptr(nb), threads)
    return dict(tau=tau, flip_mass=flip, edge_mass=edge, n_boundary=int(nb[0]))


def _forward_binned_vis(params, pts, s_begin, s_count, eps, threads, occ, eta, occ_delta):
    lib = _load()
    g = geom(params)
    P = _pts64(pts)
    S = num_scan(params)
    if s_count is None:
        s_count = S - s_begin
    if not (0 <= s_begin and s_begin + s_count <= S):
        raise ValueError("scan range out of bounds")
    B = int(params["num_bins"])
    o = occluders(occ)
    n_occ = len(np.asarray(occ).reshape(-1, 8))
    tau = np.zeros((s_count, B))
    flip = np.zeros((s_count, B)) if eps > 0 else None
    edge = np.zeros(s_count) if eps > 0 else None
    om = np.zeros((s_count, B))
    nb = np.zeros(1, dtype=np.int64)
    no = np.zeros(1, dtype=np.int64)
    lib.orc_forward_binned_vis(ctypes.byref(g), P.shape[0], _ptr(P), s_begin, s_count, o, n_occ,
                               float(eta), float(occ_delta), _ptr(tau), float(eps),
                               _ptr(flip) if flip is not None else None,
                               _ptr(edge) if edge is not None else None, _ptr(nb), _ptr(om),
                               _ptr(no), threads)
    return dict(tau=tau, flip_mass=flip, edge_mass=edge, n_boundary=int(nb[0]), occ_mass=om,
                n_occ_border=int(no[0]))


def sigma_bins(fwhm_s: float, bin_width_s: float) -> float:
    """Jitter standard deviation in bins: FWHM / (2 sqrt(2 ln 2)) / dt (Algorithm 1)."""
    return fwhm_s / (2.0 * math.sqrt(2.0 * math.log(2.0)) * bin_width_s)


def jitter_taps(fwhm_s: float, bin_width_s: float) -> np.ndarray:
    lib = _load()
    buf = np.zeros(4097)
    k = lib.orc_jitter_taps(float(fwhm_s), float(bin_width_s), _ptr(buf), buf.size)
    if k < 0:
        raise ValueError("jitter kernel too long")
    return buf[:k].copy()


PADDINGS = {"zero": 0, "replicate": 1}


def jitter(tau: np.ndarray, taps: np.ndarray, padding: str = "zero") -> np.ndarray:
    """Gaussian jitter along the last axis (Eq. 16/17) with zero padding (the
    default reading) or the edge bins replicated outside the window."""
    lib = _load()
    t = np.ascontiguousarray(tau, dtype=np.float64)
    B = t.shape[-1]
    n = t.size // B
    out = np.zeros_like(t)
    tp = np.ascontiguousarray(taps, dtype=np.float64)
    lib.orc_jitter_padded(_ptr(t), n, B, _ptr(tp), tp.size, PADDINGS[padding], _ptr(out))
    return out


def philox(ctr: np.ndarray, key) -> np.ndarray:
    """Philox4x32-10 of each counter row ([N, 4] uint32) under key (k0, k1)."""
    lib = _load()
    c = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
    k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
    out = np.zeros_like(c)
    lib.orc_philox_many(_ptr(c), c.shape[0], _ptr(k), _ptr(out))
    return out


def poisson(lam: np.ndarray, index_base: int, seed: int, stream_tag: int,
            threads: int = 0) -> np.ndarray:
    """Counts ~ Poisson(lam) from each bin's Philox stream (single precision sampler)."""
    lib = _load()
    l = np.ascontiguousarray(lam, dtype=np.float32).ravel()
    out = np.zeros(l.size, dtype=np.uint32)
    lib.orc_poisson(_ptr(l), l.size, int(index_base), int(seed) & (2**64 - 1),
                    int(stream_tag), _ptr(out), threads)
    return out.reshape(np.shape(lam))


def poisson_one(lam: float, index: int, seed: int, stream_tag: int) -> int:
    return int(_load().orc_poisson_one(float(lam), int(index), int(seed), int(stream_tag)))


def noise_lambda(tau_g: np.ndarray, params: dict):
    """Expected counts per bin, in single precision as the sampler uses them.

    peak mode (Eq. 18 with a photon budget): scale = peak_photons / max(tau_G),
    lambda = scale * tau_G + dark.  Paper mode (Eq. 18/19, Algorithm 1):
    sigma_n = Var(tau_G) / 10^(nr/10) over the whole cube (population
    variance), lambda = sigma_n * tau_G + dark (the noisy result is counts /
    sigma_n; dark counts add to lambda in both modes, a sum of Poisson
    variables being Poisson).  Both scales are taken over the whole cube given,
    not per transient."""
    t32 = np.asarray(tau_g, dtype=np.float32)
    if params["noise_mode"] == "peak":
        peak = float(np.max(t32)) if t32.size else 0.0
        scale = np.float32(params["peak_photons"]) / np.float32(peak) if peak > 0 else np.float32(0)
        dark = np.float32(params["dark_per_bin"])
    elif params["noise_mode"] == "paper_nr":
        var = float(np.var(np.asarray(tau_g, dtype=np.float64)))
        scale = np.float32(var / (10.0 ** (float(params["nr_db"]) / 10.0)))
        dark = np.float32(params["dark_per_bin"])
    else:
        raise ValueError("noise disabled")
    lam = lam_from(tau_g, scale, dark)
    return lam, float(scale), float(dark)


def lam_from(tau_g, scale, dark) -> np.ndarray:
    """lambda = fmaf(scale, float(tau_G), dark) in single precision (C fmaf)."""
    lib = _load()
    t = np.ascontiguousarray(tau_g, dtype=np.float64)
    lam = np.zeros(t.shape, dtype=np.float32)
    lib.orc_noise_lambda(_ptr(t), t.size, ctypes.c_float(scale), ctypes.c_float(dark), _ptr(lam))
    return lam


def forward_splat(params, pts, s_begin: int = 0, s_count: int | None = None,
                  threads: int = 0) -> np.ndarray:
    lib = _load()
    g = geom(params)
    P = _pts64(pts)
    S = num_scan(params)
    if s_count is None:
        s_count = S - s_begin
    B = int(params["num_bins"])
    tau = np.zeros((s_count, B))
    sg = sigma_bins(params["jitter_fwhm_s"], params["bin_width_s"])
    lib.orc_forward_splat(ctypes.byref(g), sg, P.shape[0], _ptr(P), s_begin, s_count, _ptr(tau),
                          threads)
    return tau


def backward_splat(params, pts, grad_tau: np.ndarray, threads: int = 0):
    lib = _load()
    g = geom(params)
    P = _pts64(pts)
    gt = np.ascontiguousarray(grad_tau, dtype=np.float64)
    S = num_scan(params)
    B = int(params["num_bins"])
    if gt.shape != (S, B):
        raise ValueError("grad_tau must be [S, B]")
    ga = np.zeros(P.shape[0])
    gd = np.zeros(P.shape[0])
    sg = sigma_bins(params["jitter_fwhm_s"], params["bin_width_s"])
    lib.orc_backward_splat(ctypes.byref(g), sg, P.shape[0], _ptr(P), _ptr(gt), _ptr(ga),
                           _ptr(gd), threads)
    return ga, gd


def simulate(params, pts, s_begin: int = 0, s_count: int | None = None, threads: int = 0,
             with_noise: bool = True):
    """The whole binned path for a scan range: tau, jittered tau_G, per-transient
    energy of tau_G, and (noise on) lambda and Poisson counts. The noise scale
    uses the maximum (or variance) over the scan range given, so pass the full
    scan when the scale matters."""
    r = forward_binned(params, pts, s_begin, s_count, threads=threads)
    tau = r["tau"]
    taps = jitter_taps(params["jitter_fwhm_s"], params["bin_width_s"])
    tau_g = jitter(tau, taps, params.get("jitter_padding", "zero"))
    out = dict(tau=tau, tau_g=tau_g, energy=tau_g.sum(axis=1), taps=taps)
    if with_noise and params["noise_mode"] != "none":
        lam, scale, dark = noise_lambda(tau_g, params)
        B = int(params["num_bins"])
        counts = poisson(lam, s_begin * B, params["seed"], params["stream_tag"], threads)
        out.update(lam=lam, scale=scale, dark=dark, counts=counts)
    return out
