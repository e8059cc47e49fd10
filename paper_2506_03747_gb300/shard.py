"""A transient cube split over GPUs by scan rows (one process per GPU).

Transients are independent of one another (each scan position is recorded on
its own: the paper's jitter model, Eq. 16/17, acts per scan position), so
every rank holds all surface points and simulates a contiguous block of scan
rows (``nlos_scene_create_rows``). The one dependency between ranks is the
noise scale of Eq. 18/19 (Algorithm 1 step 2.4): the maximum of the jittered
cube (PEAK) or its sum and sum of squares (PAPER_NR). Each rank reduces its
own rows (``nlos_reduce``); two all-reduces (MAX of the maxima, SUM of the
sums) give every rank the whole cube's statistics, and ``nlos_noise_part``
draws the counts from the Philox streams of the global bin indices, so the
counts do not depend on how the cube is split.

Host logic only: the row partition and the collective; every step of the
simulation runs in ``libnlos.so``.
"""
from __future__ import annotations

from . import nlos


def row_range(scan_ny: int, world: int, rank: int) -> tuple:
    """Rows [begin, begin + count) of rank `rank`: contiguous blocks whose
    sizes differ by at most one row (the first scan_ny % world ranks take the
    extra rows). count is 0 for ranks beyond scan_ny."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank must lie in [0, world)")
    base, extra = divmod(int(scan_ny), int(world))
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)


def bin_index_base(scan_nx: int, num_bins: int, row_begin: int) -> int:
    """Global index of the first bin of the part that starts at row_begin (the
    counter of its first Philox stream)."""
    return int(row_begin) * int(scan_nx) * int(num_bins)


def combine_cube_stats(stats, dist=None):
    """stats: float64 tensor [3] = {max, sum, sum of squares} of this rank's
    rows, combined in place into the whole cube's: MAX of the maxima, SUM of
    the sums (two all-reduces on the tensor's device)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return stats
    dist.all_reduce(stats[0:1], op=dist.ReduceOp.MAX)
    dist.all_reduce(stats[1:3], op=dist.ReduceOp.SUM)
    return stats


def scene_create_part(prm, points, world: int, rank: int, stream=None):
    """The scene of this rank's rows, or None for a rank without rows."""
    if isinstance(prm, dict):
        prm = nlos.params(prm)
    begin, count = row_range(prm.scan_ny, world, rank)
    if count == 0:
        return None
    return nlos.scene_create_rows(prm, points, begin, count, stream)


def simulate_part(scene, tau, counts, energy, stats, cube_bins: int, dist=None, stream=None):
    """One pass over this rank's rows: forward (pair histogram + jitter),
    per-transient energy and the rows' statistics, the all-reduce of the
    statistics, then the noise scaled by the whole cube. A rank without rows
    (scene None) joins the all-reduce with neutral statistics."""
    if scene is None:
        stats.zero_()
        combine_cube_stats(stats, dist)
        return
    nlos.forward(scene, tau, stream)
    nlos.reduce(tau, scene.num_scan, scene.num_bins, energy, stats, stream)
    combine_cube_stats(stats, dist)
    if counts is not None:
        nlos.noise_part(scene, tau, counts, stats, cube_bins, stream)
