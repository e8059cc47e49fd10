"""GPU parity of the paper's FFT forward model (nlos_lct_*, through the C ABI)
against the FP64 oracle (oracle/lct.py): random depth maps with and without
an albedo map, bins that fall outside the window, and a paper-shaped size
(128 x 128 x 1024) checked by the closed-form arrival of a plane and by
linearity."""
import numpy as np
import pytest
import torch

from oracle import lct
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


def _gpu(n, m, w, dt, depth, albedo):
    from paper_2506_03747_gb300 import nlos
    H.lib()
    plan = nlos.Lct(n, m, w, dt)
    d = torch.from_numpy(np.ascontiguousarray(depth, dtype=np.int32)).cuda()
    a = None if albedo is None else torch.from_numpy(np.ascontiguousarray(albedo, np.float32)).cuda()
    tau = torch.empty((n, n, m), dtype=torch.float32, device="cuda")
    plan.forward(d, a, tau)
    torch.cuda.synchronize()
    plan.destroy()
    return tau.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("n,m,with_albedo", [(16, 64, True), (16, 64, False), (32, 256, True),
                                             (8, 512, True)])
def test_lct_matches_oracle(n, m, with_albedo):
    rng = np.random.default_rng(n * 1000 + m)
    dt = 16e-12
    w = 0.3 * m * lct.C_LIGHT * dt   # slope 0.3
    depth = rng.integers(-3, m + 3, size=(n, n))   # some outside [0, m): no surface
    albedo = rng.random((n, n)).astype(np.float32) if with_albedo else None
    g = _gpu(n, m, w, dt, depth, albedo)
    o = lct.forward(depth, None if albedo is None else albedo.astype(np.float64), m, w, dt)
    err = np.abs(g - o)
    tol = 1e-5 * np.abs(o).max() + 1e-6 * np.abs(o)
    assert (err <= tol).all(), (err.max(), np.abs(o).max())


def test_lct_paper_shape_plane_onset_and_linearity():
    """128 x 128 depth map, 1024 bins of 32 ps (the paper's dataset shape):
    a plane at depth bin d starts, under every scan point it covers, at the
    first time bin sharing its squared-time sample; doubling the albedo
    doubles tau."""
    n, m, dt = 128, 1024, 32e-12
    w = 1.0
    d = 600
    depth = np.full((n, n), d)
    g1 = _gpu(n, m, w, dt, depth, np.full((n, n), 0.5, np.float32))
    g2 = _gpu(n, m, w, dt, depth, np.full((n, n), 1.0, np.float32))
    np.testing.assert_allclose(g2, 2 * g1, rtol=1e-6, atol=1e-6 * np.abs(g1).max())
    row = lambda j: -(-j * j // m)
    expect = min(j for j in range(1, m + 1) if row(j) == row(d + 1)) - 1
    centre = g1[n // 2, n // 2]
    # the earliest bins carry FP64 round-off of the transforms times their
    # large v^{-3/2} weights (about 1e-5 of the peak here): threshold 1e-3
    first = np.nonzero(np.abs(centre) > 1e-3 * np.abs(centre).max())[0][0]
    assert first == expect, (first, expect)
