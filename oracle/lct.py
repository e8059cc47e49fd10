"""FP64 oracle of the paper's FFT forward model (the light-cone-transform
convolution of the Theory section and Algorithm 1, steps 1.1-2.2), written
from the paper's equations with numpy and scipy.sparse. Test infrastructure:
only tests/, the smoke check and the benchmark's CPU leg use it.

Parity of this module against the paper itself is unpinned: the paper gives
no numbers for it, and several of its operators are printed ambiguously. The
readings taken (each also listed with the others of this build):

  L1 depth-to-volume (Algorithm 1, step 2.1): V[x, y, z] = albedo[x, y] at
     z = D[x, y] (0-based depth bin of a confocal N x N depth map with M
     bins), zero elsewhere; albedo in [0, 1] (the paper's A/255), 0.5 when no
     albedo map is given.
  L2 R_z (the resampling matrix): the fine matrix of M^2 rows has a nonzero
     only in rows i that are perfect squares, 1/sqrt(i) in column j = sqrt(i)
     (as printed); it is reduced to M rows by log2(M) levels of (1/2) S_k,
     S_k averaging adjacent pairs of rows, so each level scales by 1/4.
  L3 R_t^{-1}: the transpose of the fine R_z with the diagonal of
     v_i^{-3/2}, v_i = i / M^2 (the fine squared-time grid on (0, 1]), then
     the same log2(M) levels applied to its columns. The printed exponent
     +3/2 and order of the product are read as the inverse of the time
     resampling: Eq. 3 fixes v^{3/2} tau = (convolution), so the forward
     divides by v^{3/2}.
  L4 PSF (step 1.2): on the (2N) x (2N) x (2M) grid x_i, y_j, z_k in [-1, 1]
     (the printed node formulas), one nonzero per (x, y) column, at the z
     node nearest to (4 slope)^2 (x^2 + y^2), slope = w / (M c dt), when that
     value lies within half a cell of the grid; 0 elsewhere.
  L5 convolution: R_z V fills the first N x N x M corner of the zero-padded
     grid; the PSF is circularly shifted so that its node (N, N, M) (0-based:
     the first nodes above x = 0, y = 0, z = 0) sits at the origin; the
     product of the 3-D FFTs is transformed back and the first N x N x M
     corner kept; then R_t^{-1} along the last axis.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp

C_LIGHT = 299792458.0


def _levels(M: int) -> int:
    L = int(round(math.log2(M)))
    if 2 ** L != M:
        raise ValueError("the number of bins M must be a power of two")
    return L


def _half_pairs(rows: int) -> sp.csr_matrix:
    """(1/2) S_k: rows/2 x rows, entries 1/4 at columns 2i, 2i+1 (0-based)."""
    r = np.repeat(np.arange(rows // 2), 2)
    c = np.arange(rows)
    return sp.csr_matrix((np.full(rows, 0.25), (r, c)), shape=(rows // 2, rows))


def resampling_operators(M: int):
    """(R_z, R_t^{-1}), both M x M (readings L2, L3)."""
    L = _levels(M)
    n = M * M
    j = np.arange(1, M + 1)               # 1-based depth / time bins
    i = j * j                             # perfect-square fine rows
    fine = sp.csr_matrix((1.0 / np.sqrt(i), (i - 1, j - 1)), shape=(n, M))
    rz = fine
    rows = n
    for _ in range(L):
        rz = _half_pairs(rows) @ rz
        rows //= 2
    v = np.arange(1, n + 1) / float(n)
    rt = fine.T @ sp.diags(v ** -1.5)
    cols = n
    for _ in range(L):
        rt = rt @ _half_pairs(cols).T
        cols //= 2
    return rz.toarray(), rt.toarray()


def grid(n2: int) -> np.ndarray:
    """The printed nodes: -1 + 2 (i - 1) / (n2 - 1), i = 1..n2."""
    return -1.0 + 2.0 * np.arange(n2) / (n2 - 1)


def psf(N: int, M: int, wall_half: float, bin_width_s: float) -> np.ndarray:
    """PSF on the (2N, 2N, 2M) grid (reading L4)."""
    slope = wall_half / (M * C_LIGHT * bin_width_s)
    x = grid(2 * N)
    z = grid(2 * M)
    dz = z[1] - z[0]
    target = (4.0 * slope) ** 2 * (x[:, None] ** 2 + x[None, :] ** 2)
    k = np.rint((target - z[0]) / dz).astype(np.int64)
    ok = (k >= 0) & (k < 2 * M) & (np.abs(target - (z[0] + k * dz)) <= 0.5 * dz + 1e-12)
    out = np.zeros((2 * N, 2 * N, 2 * M))
    ii, jj = np.nonzero(ok)
    out[ii, jj, k[ok]] = 1.0
    return out


def volume(depth: np.ndarray, albedo: np.ndarray | None, M: int) -> np.ndarray:
    """V[x, y, z] (reading L1)."""
    N = depth.shape[0]
    d = np.asarray(depth).astype(np.int64)
    a = np.full((N, N), 0.5) if albedo is None else np.asarray(albedo, dtype=np.float64)
    V = np.zeros((N, N, M))
    ok = (d >= 0) & (d < M)
    ii, jj = np.nonzero(ok)
    V[ii, jj, d[ok]] = a[ok]
    return V


def forward(depth: np.ndarray, albedo: np.ndarray | None, M: int, wall_half: float,
            bin_width_s: float) -> np.ndarray:
    """tau[x', y', t] = R_t^{-1} F^{-1}[F(R_z V) F(PSF)] (reading L5), [N, N, M]."""
    N = depth.shape[0]
    rz, rt = resampling_operators(M)
    V = volume(depth, albedo, M)
    U = V @ rz.T                                   # resample z -> u along the last axis
    big = np.zeros((2 * N, 2 * N, 2 * M))
    big[:N, :N, :M] = U
    P = np.roll(psf(N, M, wall_half, bin_width_s), shift=(-N, -N, -M), axis=(0, 1, 2))
    conv = np.fft.ifftn(np.fft.fftn(big) * np.fft.fftn(P)).real[:N, :N, :M]
    return conv @ rt.T                             # v -> t along the last axis


def forward_direct_conv(depth, albedo, M, wall_half, bin_width_s) -> np.ndarray:
    """The same model with the 3-D convolution summed directly over the PSF's
    nonzeros (no FFT); for small grids (tests)."""
    N = depth.shape[0]
    rz, rt = resampling_operators(M)
    U = volume(depth, albedo, M) @ rz.T
    P = psf(N, M, wall_half, bin_width_s)
    conv = np.zeros((N, N, M))
    pi, pj, pk = np.nonzero(P)
    for a, b, c in zip(pi - N, pj - N, pk - M):   # PSF offsets from node (N, N, M)
        xs = slice(max(0, -a), min(N, N - a))
        ys = slice(max(0, -b), min(N, N - b))
        zs = slice(max(0, -c), min(M, M - c))
        xd = slice(xs.start + a, xs.stop + a)
        yd = slice(ys.start + b, ys.stop + b)
        zd = slice(zs.start + c, zs.stop + c)
        conv[xd, yd, zd] += U[xs, ys, zs]
    return conv @ rt.T
