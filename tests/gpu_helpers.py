"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
(via the ctypes binding) and compare it with the FP64 oracle.

Tolerances (stated by the task for this simulator):
  per bin   |tau_gpu - tau_orc| <= 1e-4 * max_b tau_orc[s, :]   (every transient s)
  energy    |E_gpu - E_orc|     <= 1e-6 * E_orc                 (every transient s)
after accounting for pairs whose bin legitimately differs between the FP32
kernel and the FP64 oracle because their path-bin coordinate u lies within
the FP32 error bound (U_EPS bins) of a bin edge.
"""
import numpy as np
import torch

import oracle
from paper_2506_03747_gb300 import build as nbuild
from paper_2506_03747_gb300 import nlos

REL_BIN = 1e-4
REL_ENERGY = 1e-6
U_EPS = 1e-3  # bound on |u_fp32 - u_fp64| in bins for windows up to 1024 bins


def u_eps(num_bins: int) -> float:
    """FP32 bound on the bin coordinate: a few ulp of the largest |u| the path
    can reach inside the window, never below U_EPS."""
    return U_EPS * max(1.0, num_bins / 1024.0)


def lib():
    nbuild.build()
    return nlos.load()


def gpu_forward(params, pts, energy=True, counts=False, stats=False, boundary_eps=0.0):
    lib()
    prm = nlos.params(params, boundary_eps=boundary_eps)
    sc = nlos.scene_create(prm, pts)
    S, B = sc.num_scan, sc.num_bins
    tau = torch.empty((S, B), dtype=torch.float32, device="cuda")
    en = torch.empty(S, dtype=torch.float64, device="cuda") if energy else None
    cn = torch.empty((S, B), dtype=torch.int32, device="cuda") if counts else None
    st = nlos.simulate(sc, tau, cn, en, stats=stats)
    torch.cuda.synchronize()
    out = dict(tau=tau.cpu().numpy().astype(np.float64), scene=sc, stats=st)
    if energy:
        out["energy"] = en.cpu().numpy()
    if counts:
        out["counts"] = cn.cpu().numpy().view(np.uint32)
    return out


def gpu_pair_table(scene, s_begin, s_count):
    P = scene.num_points
    u = torch.empty((s_count, P), dtype=torch.float32, device="cuda")
    w = torch.empty((s_count, P), dtype=torch.float32, device="cuda")
    nlos.pair_table(scene, s_begin, s_count, u, w)
    torch.cuda.synchronize()
    return u.cpu().numpy(), w.cpu().numpy()


def check_bins(tau_gpu, tau_orc, allow=None, rel=REL_BIN, what=""):
    """Per-bin rule; ``allow`` adds a per-bin allowance (flip mass)."""
    peak = tau_orc.max(axis=1, keepdims=True)
    tol = np.broadcast_to(rel * peak + (allow if allow is not None else 0.0), tau_orc.shape)
    err = np.abs(tau_gpu - tau_orc)
    bad = err > tol + 1e-30
    if bad.any():
        s, b = np.argwhere(bad)[0]
        raise AssertionError(
            f"{what}: {bad.sum()} bins out of tolerance; first s={s} b={b} gpu={tau_gpu[s, b]!r} "
            f"orc={tau_orc[s, b]!r} tol={tol[s, b]!r} peak={peak[s, 0]!r}")
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.where(peak > 0, err / peak, 0.0)
    return float(r.max()) if r.size else 0.0


def check_energy(e_gpu, e_orc, allow=None, rel=REL_ENERGY, what=""):
    tol = rel * np.abs(e_orc) + (allow if allow is not None else 0.0)
    err = np.abs(e_gpu - e_orc)
    bad = err > tol + 1e-300
    if bad.any():
        s = int(np.argwhere(bad)[0][0])
        raise AssertionError(f"{what}: energy of {bad.sum()} transients out of tolerance; "
                             f"s={s} gpu={e_gpu[s]!r} orc={e_orc[s]!r} tol={tol[s]!r}")
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.where(e_orc > 0, err / e_orc, 0.0)
    return float(r.max()) if r.size else 0.0


def flip_corrected_oracle(params, pts, scene, s_begin, s_count):
    """Oracle tau for a scan range with every pair put in the bin the GPU chose
    (after checking that each such pair is within U_EPS of a bin edge), plus the
    flip statistics and max |u32 - u64|."""
    B = int(params["num_bins"])
    u64, w64 = oracle.pair_table(params, pts, np.arange(s_begin, s_begin + s_count))
    u32, _ = gpu_pair_table(scene, s_begin, s_count)
    b64 = np.floor(u64)
    b32 = np.floor(u32.astype(np.float64))
    in64 = (u64 >= 0) & (u64 < B)
    in32 = (b32 >= 0) & (b32 < B)
    flip = (b64 != b32) & (in64 | in32)
    m = np.floor(u64 + 0.5)
    near = np.abs(u64 - m) < u_eps(B)
    assert not (flip & ~near).any(), "a pair changed bin without being near an edge"
    assert (np.abs(b64 - b32)[flip] <= 1).all()
    tau = np.zeros((s_count, B))
    for i in range(s_count):
        sel = in32[i] & (w64[i] != 0)
        np.add.at(tau[i], b32[i][sel].astype(np.int64), w64[i][sel])
    du = np.abs(u32.astype(np.float64) - u64)
    finite = np.isfinite(du) & (np.abs(u64) < 1e6)
    return tau, int(flip.sum()), float(du[finite].max()) if finite.any() else 0.0


def oracle_with_allowance(params, pts, s_begin=0, s_count=None, threads=0):
    r = oracle.forward_binned(params, pts, s_begin, s_count, eps=u_eps(int(params["num_bins"])),
                              threads=threads)
    taps = oracle.jitter_taps(params["jitter_fwhm_s"], params["bin_width_s"])
    pad = params.get("jitter_padding", "zero")
    return dict(tau=r["tau"], flip=r["flip_mass"], edge=r["edge_mass"], taps=taps, pad=pad,
                tau_g=oracle.jitter(r["tau"], taps, pad),
                flip_g=oracle.jitter(r["flip_mass"], taps, pad), n_boundary=r["n_boundary"])
