"""Pins of the FFT light-cone forward oracle (oracle/lct.py) against what the
paper's equations and plain mathematics fix: the FFT product equals the
convolution summed directly over the PSF's nonzeros, the resampling
operators' closed forms, the PSF's one-node-per-column structure and mirror
symmetry, and the arrival time of a fronto-parallel plane (t = 2 z / c)."""
import numpy as np
import pytest

from oracle import lct


@pytest.mark.parametrize("M", [4, 8, 64])
def test_resampling_operators_closed_form(M):
    rz, rt = lct.resampling_operators(M)
    assert rz.shape == (M, M) and rt.shape == (M, M)
    ez = np.zeros((M, M))
    et = np.zeros((M, M))
    for j in range(1, M + 1):
        r = -(-j * j // M) - 1          # the row block holding fine row j^2
        ez[r, j - 1] = 1.0 / (j * M * M)
        et[j - 1, r] = M / j ** 4       # (1/j) (M^2/j^2)^{3/2} / M^2
    np.testing.assert_allclose(rz, ez, rtol=1e-13, atol=0)
    np.testing.assert_allclose(rt, et, rtol=1e-13, atol=0)


def test_psf_structure():
    N, M, dt = 8, 32, 16e-12
    w = 0.2 * M * lct.C_LIGHT * dt          # slope 0.2: the cone leaves the grid at r ~ 1.25
    P = lct.psf(N, M, w, dt)
    assert P.shape == (2 * N, 2 * N, 2 * M)
    per_col = P.sum(axis=2)
    assert per_col.max() == 1.0 and per_col.sum() > N * N   # at most one node per column
    np.testing.assert_array_equal(P, P[::-1, :, :])        # x -> -x
    np.testing.assert_array_equal(P, P.transpose(1, 0, 2))  # x <-> y
    # the node of each column is the one nearest (4 slope)^2 (x^2 + y^2)
    slope = w / (M * lct.C_LIGHT * dt)
    x, z = lct.grid(2 * N), lct.grid(2 * M)
    for i in range(2 * N):
        for j in range(2 * N):
            ks = np.nonzero(P[i, j])[0]
            t = (4 * slope) ** 2 * (x[i] ** 2 + x[j] ** 2)
            if ks.size:
                assert abs(z[ks[0]] - t) <= 0.5 * (z[1] - z[0]) + 1e-12
            else:
                assert t > z[-1]


def test_fft_equals_direct_convolution():
    rng = np.random.default_rng(2)
    N, M, w, dt = 6, 16, 0.4, 12e-12
    depth = rng.integers(0, M, size=(N, N))
    albedo = rng.random((N, N))
    a = lct.forward(depth, albedo, M, w, dt)
    b = lct.forward_direct_conv(depth, albedo, M, w, dt)
    assert a.shape == (N, N, M)
    np.testing.assert_allclose(a, b, rtol=1e-10, atol=1e-12 * np.abs(b).max())
    # linear in the albedo; no albedo map = 0.5 everywhere
    np.testing.assert_allclose(lct.forward(depth, 2 * albedo, M, w, dt), 2 * a, rtol=1e-12,
                               atol=1e-15)
    np.testing.assert_allclose(lct.forward(depth, None, M, w, dt),
                               lct.forward(depth, np.full((N, N), 0.5), M, w, dt), rtol=1e-12,
                               atol=0)


def test_plane_arrival_time():
    """A fronto-parallel plane at depth bin d (z = (d + 1) c dt / 2): the
    centre transient starts at t = 2 z / c, i.e. at the first time bin that
    shares the plane's squared-time sample (the model resamples depth and time
    onto M samples of z^2 and t^2: ceil(j^2 / M) groups the 1-based bins j)."""
    N, M, dt = 16, 64, 16e-12
    w = 0.5 * N * lct.C_LIGHT * dt / 2   # scan pitch = c dt / 2 (square voxels)
    row = lambda j: -(-j * j // M)       # ceil(j^2 / M), 1-based bin j
    for d in [10, 25, 40]:
        depth = np.full((N, N), d)
        # the direct sum over the PSF: exact zeros before the onset (the FFT's
        # round-off is amplified by the v^{-3/2} weight of the earliest bins)
        tau = lct.forward_direct_conv(depth, None, M, w, dt)
        first = np.nonzero(tau[N // 2, N // 2])[0][0]
        expect = min(j for j in range(1, M + 1) if row(j) == row(d + 1)) - 1
        assert first == expect, (d, first, expect)
        assert expect <= d


def test_agrees_with_the_direct_sum():
    """The FFT model approximates Eq. 1 itself (its defining integral): on a
    tilted plane with random albedo, sampled at the depth-bin centres of the
    same scan grid, the cubes correlate above 0.85 (0.90 measured) and the
    per-transient energies above 0.9 (0.95): the model resamples depth and
    time onto M samples of z^2 and t^2, which smears early bins. Only the
    shape is compared (the model's scale is a convention)."""
    import oracle
    import scenes
    N, M, dt = 32, 128, 16e-12
    cdt2 = lct.C_LIGHT * dt / 2
    w = N * cdt2
    pitch = 2 * w / N
    rng = np.random.default_rng(0)
    xs = -w + (np.arange(N) + 0.5) * pitch
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    d = np.clip(np.rint((0.4 * M * cdt2 + 0.15 * X + 0.05 * Y) / cdt2 - 1).astype(int), 0, M - 1)
    alb = 0.3 + 0.7 * rng.random((N, N))
    t_lct = lct.forward(d, alb, M, w, dt)
    pts = np.zeros((N * N, 8), np.float32)
    pts[:, 0], pts[:, 1], pts[:, 2] = X.ravel(), Y.ravel(), ((d + 1) * cdt2).ravel()
    pts[:, 5], pts[:, 6], pts[:, 7] = -1.0, alb.ravel(), pitch * pitch
    params = scenes.default_params(scan_nx=N, scan_ny=N, wall_half_x=w, wall_half_y=w,
                                   bin_width_s=dt, num_bins=M, window_start_m=0.0,
                                   cos_mode="none")
    t_dir = oracle.forward_binned(params, pts)["tau"].reshape(N, N, M).transpose(1, 0, 2)
    a, b = t_lct.ravel(), t_dir.ravel()
    assert (a @ b) / np.linalg.norm(a) / np.linalg.norm(b) > 0.85
    assert np.corrcoef(t_lct.sum(-1).ravel(), t_dir.sum(-1).ravel())[0, 1] > 0.9
