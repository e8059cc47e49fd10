"""A cube split by scan rows on one GPU: the parts (nlos_scene_create_rows)
simulated one after the other, their statistics combined as the ranks'
all-reduces would (max of the maxima, sums of the sums), and the noise of each
part drawn with the whole cube's scale (nlos_noise_part). The concatenated
parts match the whole scene: transients at the parity bar, counts equal but
where lambda differs in its last bits, and both against the oracle."""
import numpy as np
import pytest
import torch

import oracle
import scenes
from tests import gpu_helpers as H

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode,world", [("peak", 2), ("paper_nr", 3)])
def test_split_cube_matches_whole(mode, world):
    from paper_2506_03747_gb300 import nlos, shard
    H.lib()
    rng = np.random.default_rng(5)
    pts = scenes.random_points(rng, 3001, half=0.6, z_lo=0.3, z_hi=1.1)
    params = scenes.default_params(scan_nx=19, scan_ny=13, wall_half_x=0.7, wall_half_y=0.6,
                                   scan_mode="nonconfocal", laser_xy=(0.1, -0.05),
                                   bin_width_s=8e-12, num_bins=400, jitter_fwhm_s=50e-12,
                                   standoff_m=0.3, standoff_mode="euclidean", noise_mode=mode,
                                   peak_photons=100.0, dark_per_bin=1e-3, nr_db=2.0, seed=9)
    nx, ny, B = params["scan_nx"], params["scan_ny"], params["num_bins"]
    whole = H.gpu_forward(params, pts, counts=True, stats=True)
    pd = torch.from_numpy(pts).cuda()
    parts = []
    stats_all = []
    for r in range(world):
        sc = shard.scene_create_part(params, pd, world, r)
        S = sc.num_scan
        tau = torch.empty((S, B), dtype=torch.float32, device="cuda")
        en = torch.empty(S, dtype=torch.float64, device="cuda")
        st = torch.empty(3, dtype=torch.float64, device="cuda")
        nlos.forward(sc, tau)
        nlos.reduce(tau, S, B, en, st)
        parts.append((sc, tau, en))
        stats_all.append(st)
    cube = torch.stack(stats_all)
    cube = torch.stack([cube[:, 0].max(), cube[:, 1].sum(), cube[:, 2].sum()]).contiguous()
    counts = []
    for sc, tau, _ in parts:
        c = torch.empty((sc.num_scan, B), dtype=torch.int32, device="cuda")
        nlos.noise_part(sc, tau, c, cube, nx * ny * B)
        counts.append(c)
    torch.cuda.synchronize()
    tau_cat = np.concatenate([t.cpu().numpy().astype(np.float64) for _, t, _ in parts])
    en_cat = np.concatenate([e.cpu().numpy() for _, _, e in parts])
    cnt_cat = np.concatenate([c.cpu().numpy().view(np.uint32) for c in counts])
    # the parts' rows in order give the whole cube
    assert tau_cat.shape == whole["tau"].shape
    H.check_bins(tau_cat, whole["tau"], rel=1e-5, what="parts vs whole")
    H.check_energy(en_cat, whole["energy"], rel=1e-6, what="parts vs whole energy")
    diff = int((cnt_cat != whole["counts"]).sum())
    assert diff <= max(2, cnt_cat.size // 10000), diff
    # and the parts against the oracle at the parity bars
    o = H.oracle_with_allowance(params, pts)
    H.check_bins(tau_cat, o["tau_g"], allow=o["flip_g"], what="parts vs oracle")
    for sc, _, _ in parts:
        sc.destroy()
