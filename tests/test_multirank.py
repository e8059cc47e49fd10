"""Multi-rank logic on CPU with two gloo ranks.

* bench.py: the whole-job rate is all ranks' units over the slowest rank's
  time; independent scenes get distinct seeds.
* A cube split over ranks by scan rows (paper_2506_03747_gb300.shard): each
  rank computes its rows (here with the FP64 oracle standing in for the CUDA
  kernels, which need a GPU), the ranks combine the rows' statistics with the
  same all-reduces the GPU path uses, and draw the noise from the Philox
  streams of the global bin indices; the concatenated transients and counts
  equal the single-rank result bit for bit."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench._dist()
    seconds = 1.0 + rank  # rank 1 is the slow one
    rate, t = bench.whole_job_rate(100.0, seconds, ws, dist, "cpu")
    q.put((rank, ws, r, local, bench.workload_seed("heightfield128", rank), rate, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_rate_and_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    (r0, ws0, rr0, l0, seed0, rate0, t0), (r1, ws1, rr1, l1, seed1, rate1, t1) = res
    assert ws0 == ws1 == 2 and (rr0, rr1) == (0, 1) and (l0, l1) == (0, 1)
    assert seed0 != seed1
    # max over ranks: both see the slow rank's 2 s; whole job = 2 x 100 units / 2 s
    assert t0 == t1 == 2.0
    assert rate0 == rate1 == pytest.approx(100.0)


def test_single_rank_rate():
    import bench
    rate, t = bench.whole_job_rate(50.0, 0.5, 1)
    assert (rate, t) == (100.0, 0.5)


def _split_rank_main(rank, world, port, q, mode):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import numpy as np
    import oracle
    import scenes
    from paper_2506_03747_gb300 import shard
    params, pts = _split_case(mode)
    nx, ny, B = params["scan_nx"], params["scan_ny"], params["num_bins"]
    begin, count = shard.row_range(ny, world, rank)
    # this rank's rows, as the forward + jitter of its part compute them
    r = oracle.forward_binned(params, pts, begin * nx, count * nx)
    taps = oracle.jitter_taps(params["jitter_fwhm_s"], params["bin_width_s"])
    tau_g = oracle.jitter(r["tau"], taps)
    stats = torch.tensor([tau_g.max(), tau_g.sum(), (tau_g * tau_g).sum()], dtype=torch.float64)
    shard.combine_cube_stats(stats, dist)
    mx, sm, sq = (float(v) for v in stats)
    n = nx * ny * B
    if mode == "peak":
        scale = np.float32(params["peak_photons"]) / np.float32(mx)
    else:
        var = sq / n - (sm / n) ** 2
        scale = np.float32(var / 10.0 ** (params["nr_db"] / 10.0))
    lam = oracle.lam_from(tau_g, float(scale), float(np.float32(params["dark_per_bin"])))
    counts = oracle.poisson(lam, shard.bin_index_base(nx, B, begin), params["seed"],
                            params["stream_tag"])
    q.put((rank, begin, count, tau_g, counts, float(scale)))
    dist.barrier()
    dist.destroy_process_group()


def _split_case(mode):
    import numpy as np
    import scenes
    rng = np.random.default_rng(31)
    pts = scenes.random_points(rng, 700, half=0.5, z_lo=0.3, z_hi=1.0)
    params = scenes.default_params(scan_nx=9, scan_ny=7, wall_half_x=0.6, wall_half_y=0.5,
                                   bin_width_s=8e-12, num_bins=300, jitter_fwhm_s=50e-12,
                                   standoff_m=0.2, standoff_mode="euclidean",
                                   noise_mode=mode, peak_photons=100.0, dark_per_bin=1e-3,
                                   nr_db=2.0, seed=77, stream_tag=3)
    return params, pts


@pytest.mark.parametrize("mode", ["peak", "paper_nr"])
def test_split_cube_two_ranks_equals_one_rank(mode):
    import numpy as np
    import oracle
    from paper_2506_03747_gb300 import shard
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_rank_main, args=(r, 2, port, q, mode)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in range(2)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    params, pts = _split_case(mode)
    nx, ny = params["scan_nx"], params["scan_ny"]
    # the parts tile the rows exactly once, in order
    assert [(b, c) for _, b, c, _, _, _ in res] == [shard.row_range(ny, 2, 0), shard.row_range(ny, 2, 1)]
    assert res[0][1] == 0 and res[0][1] + res[0][2] == res[1][1] and res[1][1] + res[1][2] == ny
    whole = oracle.simulate(params, pts)
    np.testing.assert_array_equal(np.concatenate([r[3] for r in res]), whole["tau_g"])
    np.testing.assert_array_equal(np.concatenate([r[4] for r in res]), whole["counts"])
    assert res[0][5] == res[1][5] == pytest.approx(whole["scale"], rel=1e-6)


def test_row_range_partitions():
    from paper_2506_03747_gb300 import shard
    for ny in (1, 7, 128, 129):
        for world in (1, 2, 3, 8):
            parts = [shard.row_range(ny, world, r) for r in range(world)]
            assert sum(c for _, c in parts) == ny
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
            pos = 0
            for b, c in parts:
                assert b == pos or c == 0
                pos += c
    assert shard.bin_index_base(128, 1024, 64) == 64 * 128 * 1024
