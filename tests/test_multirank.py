"""The multi-rank logic of bench.py on CPU with two gloo ranks: every rank
processes its own independent scene (distinct seeds, same workload shape), and
the whole-job rate is all ranks' units over the slowest rank's time."""
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
    q.put((rank, ws, r, local, bench.workload_seed(rank), rate, t))
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
