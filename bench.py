#!/usr/bin/env python
"""Benchmark of the GB300 NLOS transient simulator.

Metric: pair-interactions/s of the whole forward hot path (ingest/pack,
pair histogram with fused jitter, FP64 energy reduction, Philox Poisson
noise), inputs resident in HBM, on the largest single-GPU workload: the
non-confocal 128x128-scan heightfield (1,048,576 surface points, 1024 bins of
4 ps, 1.5 m stand-off, 30 ps jitter, 100-photon peak + 1e-3 dark counts;
1.72e10 pairs per pass). The confocal union-of-primitives workload (64x64
scan, 262,144 points, 512 bins of 8 ps) is reported beside it under
"union64". One JSON line on rank 0; see --help.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun (N > 1) the ranks share one cube split by scan rows (every
rank holds all points and simulates its block of rows; one all-reduce of the
cube's max / sums before the noise): strong scaling. With --replicas every
rank simulates its own independent scene instead (seed offset by the rank):
weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "pair-interactions/s vs FP32 roofline; served p50/p99 latency vs one-by-one"
UNIT = "pairs/s"
FP32_SLOTS_PER_PAIR = 17   # algorithmic FP32 issue slots per evaluated pair
FP32_SLOTS_EARLY_OUT = 6   # slots of a pair stopped by the early out (dx, dy, r^2, cosine)
MUFU_PER_PAIR = 2          # square root and reciprocal estimates per evaluated pair
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
HEADLINE = "heightfield128"
WORKLOAD_DESC = {
    "heightfield128": (
        "heightfield128: non-confocal (laser at the wall centre) 128x128 detector scan over "
        "2 m x 2 m, 1024 bins x 4 ps, stand-off 1.5 m (Euclidean legs), acquisition window from "
        "L0 = 3.8 m (2 x 1.5 m + 2 x 0.4 m: the earliest round trip from the wall centre), "
        "1,048,576 points of a seeded 1024x1024 heightfield at 0.4-1.5 m, albedo Beta(2,2), "
        "jitter FWHM 30 ps, Poisson noise peak 100 photons + 1e-3 dark/bin"),
    "union64": (
        "union64: confocal 64x64 scan over 2 m x 2 m, 512 bins x 8 ps, stand-off 1 m "
        "(Euclidean legs), acquisition window from L0 = 2.6 m (2 x 1 m + 2 x 0.3 m), "
        "262,144 area-uniform points on a seeded union of 3-6 spheres/boxes at 0.3-1.2 m, "
        "albedo U[0.2,1], jitter FWHM 60 ps, Poisson noise peak 100 photons + 1e-3 dark/bin"),
}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def whole_job_rate(units_per_rank: float, seconds: float, world_size: int, dist=None,
                   device=None) -> tuple:
    """Weak scaling with independent problems: every rank processes the same
    number of units; the job takes as long as its slowest rank (max over ranks
    of the timed seconds), and the whole-job rate is all ranks' units over that
    time. Returns (rate, max_seconds)."""
    t = seconds
    if dist is not None and world_size > 1:
        import torch
        x = torch.tensor([seconds], dtype=torch.float64, device=device)
        dist.all_reduce(x, op=dist.ReduceOp.MAX)
        t = float(x.item())
    return world_size * units_per_rank / t, t


def workload_seed(name: str, rank: int) -> int:
    """Each rank simulates its own independent scene of the same workload."""
    import scenes
    return scenes.SEED_BASE + (3 if name == "heightfield128" else 2) + 1000 * rank


def _workload(name: str, rank: int):
    import scenes
    fn = scenes.workload_heightfield128 if name == "heightfield128" else scenes.workload_union64
    return fn(seed=workload_seed(name, rank))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        # raw samples: a temporary file, or the directory NLOS_BENCH_CLOCKS_DIR names
        self.path = os.path.join(os.environ.get("NLOS_BENCH_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                c = [x.strip() for x in line.split(",")]
                if len(c) < 9:
                    continue
                try:
                    sm.append(float(c[1]))
                    smax.append(float(c[2]))
                except ValueError:
                    continue
                for n, v in zip(names, c[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)),
                "reasons": sorted(reasons), "samples": len(sm)}


FORWARD_SOURCES = ("forward.cu", "forward_core.cuh", "device_util.cuh", "common.cuh")
# FP32 issue slots per (scan point, point) pair of the moment-form adjoint
# kernel, counted from its source: per leg the differences, squared length
# and square root (2 + 3 + 4), the normal's dot product (3), the reciprocal,
# cosine, its derivative and the 1/r^2 factor (18), 30 a leg; then the weight
# and its two derivatives (8), u and du/d(delta) (4), the moment row and c (5),
# two 6-term Horner evaluations and G1 (12), the two products (4), 33 in all.
# A pair evaluates one leg: a confocal scan's laser spot is its detector spot,
# and a non-confocal scan's laser leg depends on the point only (the kernel
# computes it once per point): 63 (a few of these are integer or select
# instructions).
ADJ_FP32_SLOTS_PER_PAIR = {"confocal": 63, "nonconfocal": 63}


def launches_per_step(split: bool) -> int:
    """Kernels of this library one bench step launches: the ingest (counts and
    box initialised, bounding box, Morton cells, the scan of the cell counts,
    the scatter, pack + block bounds), the forward (live-unit list, pair
    histogram), and the detect step (reduce; noise and its second pass over the
    deferred bright bins); a split cube reduces through nlos_reduce, which adds
    the statistics copy kernel."""
    return 6 + 2 + (4 if split else 3)


def forward_sources_sha256() -> str:
    """One SHA-256 over the sources the forward kernel is compiled from."""
    h = hashlib.sha256()
    for name in FORWARD_SOURCES:
        with open(os.path.join(ROOT, "paper_2506_03747_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _traffic_for(name: str):
    """DRAM bytes per forward launch from the committed ncu summary of this
    workload, if it was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", f"forward_{name}_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    ok = d.get("forward_sources_sha256") == forward_sources_sha256()
    return d.get("dram_bytes_per_launch") if ok else None


def _sample_range(S: int, count: int) -> tuple:
    """A contiguous block of scan points around the middle of the scan (the
    oracle's cost per pair does not depend on which)."""
    count = max(1, min(S, count))
    begin = max(0, S // 2 - count // 2)
    return begin, count


def cpu_baseline(params, pts, scan_count: int):
    """The FP64 oracle as it stands, on all host cores, on a block of
    scan_count scan points of the workload (forward + jitter + energy +
    noise); pairs/s of that sample."""
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    S = params["scan_nx"] * params["scan_ny"]
    s0, n = _sample_range(S, scan_count)
    t0 = time.perf_counter()
    oracle.simulate(params, pts, s0, n, threads=cores)
    dt = time.perf_counter() - t0
    pairs = n * pts.shape[0]
    return {"value": pairs / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"scan points {s0}..{s0 + n - 1} of {S} x all {pts.shape[0]} points, one "
                      f"pass (FP64 forward + jitter + energy + Poisson noise), {dt:.2f} s wall"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    params, pts = _workload(HEADLINE, 0)
    S = params["scan_nx"] * params["scan_ny"]
    s0, n = _sample_range(S, args.ref_scan)  # bounded sample per step
    import oracle
    oracle.build()
    cores = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.simulate(params, pts, s0, n, threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.simulate(params, pts, s0, n, threads=cores)
    dt = time.perf_counter() - t0
    pairs = args.steps * n * pts.shape[0]
    v = pairs / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD_DESC[HEADLINE],
                                            "sample_per_step": f"{n} of {S} scan points"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"scan points {s0}..{s0 + n - 1} of {S} x "
                                       f"{pts.shape[0]} points per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def device_peaks():
    """Measured element rates per SM clock (nlos_measure_peaks), or None."""
    from paper_2506_03747_gb300 import nlos
    try:
        return nlos.measure_peaks()
    except Exception:  # measurement only; the roofline then says so
        return None


def forward_roofline(name, fwd_s, st, pairs_per_step, n_sm, sm_max_mhz, peaks, S, B):
    """Roofline of the pair-histogram kernel: evaluated pairs (full-evaluation
    equivalents) per second against the binding one of the FP32 pipe (17
    slots per pair) and the MUFU pipe (2 estimates per pair) at the measured
    per-SM rates and the maximum SM clock."""
    f = sm_max_mhz * 1e6
    if peaks:
        ffma, mufu, basis = peaks["ffma"], peaks["sqrt_approx"], "measured (nlos_measure_peaks)"
    else:
        ffma, mufu, basis = 128.0, 16.0, "nominal (128 FP32 lanes, 16 MUFU lanes per SM clock)"
    fp32_peak = n_sm * ffma * f / FP32_SLOTS_PER_PAIR
    mufu_peak = n_sm * mufu * f / MUFU_PER_PAIR
    peak = min(fp32_peak, mufu_peak)
    full, tested = int(st["pairs_full"]), int(st["pairs_tested"])
    # pairs of culled units cost nothing per pair and are not counted as work
    work = full + max(0, tested - full) * FP32_SLOTS_EARLY_OUT / FP32_SLOTS_PER_PAIR
    achieved = work / fwd_s
    return {"bound": "alu", "achieved": achieved / 1e9, "peak": peak / 1e9, "unit": "Gpair/s",
            "frac": achieved / peak, "traffic": _traffic_for(name),
            "kernel": "fwd_kernel (pair histogram + fused jitter)",
            "peak_basis": f"min(FP32: {n_sm} SMs x {ffma:.1f} FMA lanes/clk x {sm_max_mhz:.0f} MHz / "
                          f"{FP32_SLOTS_PER_PAIR} slots per pair = {fp32_peak / 1e9:.0f} Gpair/s; "
                          f"MUFU: {n_sm} x {mufu:.1f} lanes/clk x {sm_max_mhz:.0f} MHz / "
                          f"{MUFU_PER_PAIR} per pair = {mufu_peak / 1e9:.0f} Gpair/s), {basis}",
            "work_basis": f"full-evaluation-equivalent pairs: pairs evaluated in full + "
                          f"{FP32_SLOTS_EARLY_OUT}/{FP32_SLOTS_PER_PAIR} x pairs stopped by "
                          f"the early out; pairs of units ruled out by the block bounds "
                          f"count 0",
            "pairs_full_fraction": full / pairs_per_step,
            "pairs_tested_fraction": tested / pairs_per_step,
            "effective_pairs_per_s": pairs_per_step / fwd_s,
            "kernel_ms": fwd_s * 1e3,
            "tau_write_gbs": S * B * 4 / fwd_s / 1e9}


def measure_workload(name, rank, steps, warmup, local, dist, ws, peaks, clocks=None,
                     split=False):
    """Times `steps` bench steps of one workload (scene_set_points = ingest and
    pack, forward = pair histogram with fused jitter, detect = FP64 energy,
    cube statistics and Poisson noise), inputs resident in HBM, L2 flushed
    between steps; then the same steps end to end with host buffers.
    split: the ranks share one cube, each simulating its block of scan rows
    (paper_2506_03747_gb300.shard; one all-reduce of the cube statistics
    before the noise); else every rank simulates its own scene."""
    import torch
    from paper_2506_03747_gb300 import nlos, shard
    params, pts_np = _workload(name, 0 if split else rank)
    stream = torch.cuda.current_stream()
    pts_dev = torch.from_numpy(pts_np).cuda()
    if split:
        scene = shard.scene_create_part(params, pts_dev, ws, rank)
        if scene is None:
            raise RuntimeError("more ranks than scan rows")
    else:
        scene = nlos.scene_create(nlos.params(params), pts_dev)
    S, B, P = scene.num_scan, scene.num_bins, scene.num_points
    S_cube = params["scan_nx"] * params["scan_ny"]
    tau = torch.empty((S, B), dtype=torch.float32, device="cuda")
    counts = torch.empty((S, B), dtype=torch.int32, device="cuda")
    energy = torch.empty(S, dtype=torch.float64, device="cuda")
    cube_stats = torch.empty(3, dtype=torch.float64, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    # whole-job units per step and rank: a split cube is one cube over all ranks
    pairs_per_step = (S_cube * P / ws) if split else S * P

    def detect():
        if split:
            nlos.reduce(tau, S, B, energy, cube_stats)
            shard.combine_cube_stats(cube_stats, dist)
            nlos.noise_part(scene, tau, counts, cube_stats, S_cube * B)
        else:
            nlos.detect(scene, tau, counts, energy)

    def step():
        nlos.scene_set_points(scene, pts_dev)
        nlos.forward(scene, tau)
        detect()

    for _ in range(max(3, warmup)):
        step()
    nlos.scene_check(scene)
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
        time.sleep(0.3)
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for k in range(steps):
        flush.zero_()  # evict L2 between timed steps (outside the step events)
        e = ev[k]
        e[0].record(stream)
        nlos.scene_set_points(scene, pts_dev)
        e[1].record(stream)
        nlos.forward(scene, tau)
        e[2].record(stream)
        detect()
        e[3].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall = time.perf_counter() - wall0
    clk = clocks.stop() if clocks else None
    nlos.scene_check(scene)
    step_ms = np.array([e[0].elapsed_time(e[3]) for e in ev])
    pack_ms = np.array([e[0].elapsed_time(e[1]) for e in ev])
    fwd_ms = np.array([e[1].elapsed_time(e[2]) for e in ev])
    det_ms = np.array([e[2].elapsed_time(e[3]) for e in ev])
    value, t_total = whole_job_rate(steps * pairs_per_step, float(step_ms.sum()) * 1e-3, ws,
                                    dist, "cuda")

    # ---- end to end through the C ABI with host buffers (pinned) ----------
    # Every step copies its points from pinned host memory (scene_set_points
    # with a host pointer) and reads its counts back; L2 is flushed before each
    # step inside the timed region. One cube per rank: two scenes on two streams
    # alternate, so one step's copies overlap the other's kernels (the time is
    # the whole run's, first step's start to last step's end). A split cube
    # (an all-reduce inside each step) runs its steps one after the other.
    pts_host = torch.from_numpy(pts_np).pin_memory()
    if split:
        counts_host = torch.empty((S, B), dtype=torch.int32).pin_memory()
        e2e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
        for _ in range(2):
            nlos.scene_set_points(scene, pts_host)
            nlos.forward(scene, tau)
            detect()
            counts_host.copy_(counts, non_blocking=True)
        torch.cuda.synchronize()
        for k in range(steps):
            flush.zero_()
            a, b = e2e_ev[k]
            a.record(stream)
            nlos.scene_set_points(scene, pts_host)          # H2D of the step's points
            nlos.forward(scene, tau)
            detect()
            counts_host.copy_(counts, non_blocking=True)    # D2H of the step's result
            b.record(stream)
        torch.cuda.synchronize()
        e2e_s = sum(a.elapsed_time(b) for a, b in e2e_ev) * 1e-3
        overlap = "none (steps in sequence)"
    else:
        scene_b = nlos.scene_create(nlos.params(params), pts_dev)
        sc2 = [scene, scene_b]
        tau2 = [tau, torch.empty_like(tau)]
        cnt2 = [counts, torch.empty_like(counts)]
        en2 = [energy, torch.empty_like(energy)]
        host2 = [torch.empty((S, B), dtype=torch.int32).pin_memory() for _ in range(2)]
        st2 = [torch.cuda.Stream(), torch.cuda.Stream()]

        def e2e_step(j, do_flush):
            with torch.cuda.stream(st2[j]):
                if do_flush:
                    flush.zero_()
                nlos.scene_set_points(sc2[j], pts_host)     # H2D of the step's points
                nlos.forward(sc2[j], tau2[j])
                nlos.detect(sc2[j], tau2[j], cnt2[j], en2[j])
                host2[j].copy_(cnt2[j], non_blocking=True)  # D2H of the step's result

        for k in range(4):
            e2e_step(k % 2, False)
        torch.cuda.synchronize()
        t0 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for s_ in st2:
            s_.wait_event(t0)
        for k in range(steps):
            e2e_step(k % 2, True)
        t1 = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
        for j in range(2):
            t1[j].record(st2[j])
        torch.cuda.synchronize()
        e2e_s = max(t0.elapsed_time(t1[j]) for j in range(2)) * 1e-3
        nlos.scene_check(scene_b)
        scene_b.destroy()
        overlap = "two scenes on two streams, alternating steps"
    e2e_rate, _ = whole_job_rate(steps * pairs_per_step, e2e_s, ws, dist, "cuda")
    e2e = {"value": e2e_rate, "unit": UNIT,
           "h2d_bytes_per_step": int(pts_np.nbytes), "d2h_bytes_per_step": int(S * B * 4),
           "overlap": overlap, "l2": "flushed before each step, inside the timed region"}

    props = torch.cuda.get_device_properties(local)
    sm_max = (clk or {}).get("sm_max_mhz") or 2070.0
    st = nlos.simulate(scene, tau, None, None, stats=True)
    roof = forward_roofline(name, float(fwd_ms.mean()) * 1e-3, st, S * P,
                            props.multi_processor_count, sm_max, peaks, S, B)
    scene.destroy()
    return {"value": value, "ms_per_step": t_total * 1e3 / steps,
            "transients_per_s": ws * steps * S / t_total, "wall_s": wall, "clocks": clk,
            "phase_ms": {"ingest_pack": float(pack_ms.mean()), "forward": float(fwd_ms.mean()),
                         "detect": float(det_ms.mean())},
            "roofline": roof, "e2e": e2e, "params": params, "pts": pts_np,
            "shape": {"scan_points": S, "bins": B, "points": P, "pairs_per_step": pairs_per_step}}


def run_ours(args):
    import torch
    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2506_03747_gb300 import build as nbuild
    from paper_2506_03747_gb300 import nlos
    nbuild.build()
    nlos.load()
    peaks = device_peaks()

    split = ws > 1 and not args.replicas
    head = measure_workload(HEADLINE, rank, args.steps, args.warmup, local, dist, ws, peaks,
                            clocks=ClockSampler(local), split=split)
    extra = None
    if args.union_steps > 0:
        extra = measure_workload("union64", rank, args.union_steps, args.warmup, local, dist, ws,
                                 peaks, split=split)
    line = {"metric": METRIC, "value": head["value"], "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": head["ms_per_step"],
            "higher_is_better": True, "scaling": "strong" if split else "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict({"workload": WORKLOAD_DESC[HEADLINE]}, **head["shape"],
                           l2="flushed by a 256 MB write between timed steps (outside the step "
                              "events)",
                           step="scene_set_points (ingest: spatial order + pack + bounds) + "
                                "forward (pair histogram + fused jitter) + detect (FP64 energy, "
                                "cube max and sums, Poisson noise)",
                           parallelism=(f"one cube split over {ws} GPUs by scan rows (all "
                                        f"points on every GPU; one all-reduce of the cube "
                                        f"statistics before the noise)") if split else
                           f"{ws} independent scenes, one per GPU"),
            "transients_per_s": head["transients_per_s"], "wall_s": head["wall_s"],
            "clocks": head["clocks"], "gpu_launches": launches_per_step(split) * args.steps,
            "phase_ms": head["phase_ms"], "roofline": head["roofline"], "e2e": head["e2e"]}
    if peaks:
        line["device_peaks_per_sm_clock"] = peaks
    if extra is not None:
        line["union64"] = {"workload": WORKLOAD_DESC["union64"], **extra["shape"],
                           "value": extra["value"], "ms_per_step": extra["ms_per_step"],
                           "phase_ms": extra["phase_ms"], "roofline": extra["roofline"],
                           "e2e": extra["e2e"]}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(head["params"], head["pts"], args.cpu_scan)
    if rank == 0 and ws == 1 and args.splat_steps > 0:
        line["splat_adjoint"] = splat_adjoint_bench(args.splat_steps, 1, peaks)
    if rank == 0 and ws == 1 and args.serving_requests > 0:
        line["serving"] = serving_bench(args.serving_requests, args.serving_rate)
    if rank == 0 and ws == 1 and args.saturate_requests > 0:
        # the same request mix arriving far faster than either mode serves it
        # (a saturating leg: throughput at full load, latency dominated by queueing)
        line["serving_saturated"] = serving_bench(args.saturate_requests, args.saturate_rate)
    if rank == 0 and ws == 1 and args.lct_steps > 0:
        line["lct"] = lct_bench(args.lct_steps, peaks)
    if rank == 0 and ws == 1 and args.occlusion_steps > 0:
        line["occlusion"] = occlusion_bench(args.occlusion_steps)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def occlusion_bench(steps: int):
    """The union workload's forward with its own spheres and boxes as
    occluders (the visibility extension: one segment test per binned pair and
    occluder) against the same forward without them; L2 flushed between
    launches. Effective pairs/s = S * P / time."""
    import torch
    import scenes
    from paper_2506_03747_gb300 import nlos
    params, _ = scenes.workload_union64()
    rng = np.random.default_rng(scenes.SEED_BASE + 2)
    pts, prims = scenes.primitive_union_points(rng, 262144)
    occ = scenes.occluder_records(prims)
    sc = nlos.scene_create(nlos.params(params), torch.from_numpy(pts).cuda())
    S, B = sc.num_scan, sc.num_bins
    tau = torch.empty((S, B), dtype=torch.float32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {}
    for name, o in (("without", None), ("with", occ)):
        nlos.scene_set_occluders(sc, o)
        for _ in range(3):
            nlos.forward(sc, tau)
        ts = []
        for _ in range(steps):
            flush.fill_(1)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            nlos.forward(sc, tau)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        out[name] = float(np.median(ts))
    sc.destroy()
    pairs = S * len(pts)
    return {"workload": f"union64 ({S} scan points x {len(pts)} points, 512 bins) with its "
                        f"{len(occ)} primitives as occluders",
            "occluders": len(occ), "forward_ms_without": out["without"],
            "forward_ms_with": out["with"],
            "effective_pairs_per_s_with": pairs / (out["with"] * 1e-3),
            "slowdown": out["with"] / out["without"]}


def lct_bench(steps: int, peaks=None):
    """The paper's FFT forward model on its dataset shape (128 x 128 depth map,
    1024 bins of 32 ps, 2 m wall) against the direct pair sum of Eq. 1 on the
    same surface (one point per pixel at its depth-bin centre, no cosines,
    window from the wall). Reports both times, the shape correlation, and the
    FFT model's FP64 roofline: two 3-D radix-2 transforms of the
    (2N) x (2N) x (2M) volume V at 5 V log2(V) flops each, and the 6 V of the
    spectral product, against the measured FP64 fma rate (2 flops each)."""
    import torch
    from paper_2506_03747_gb300 import nlos
    n, m, dt, w = 128, 1024, 32e-12, 1.0
    cdt2 = 299792458.0 * dt / 2
    rng = np.random.default_rng(0x4E4C4F53 + 9)
    xs = -w + (np.arange(n) + 0.5) * (2 * w / n)
    X, Y = np.meshgrid(xs, xs, indexing="ij")
    z = 0.8 + 0.3 * np.exp(-((X - 0.2) ** 2 + Y ** 2) / 0.1) + 0.1 * X
    depth = np.clip(np.rint(z / cdt2 - 1).astype(np.int32), 0, m - 1)
    albedo = (0.2 + 0.8 * rng.beta(2, 2, size=(n, n))).astype(np.float32)
    d_dev = torch.from_numpy(depth).cuda()
    a_dev = torch.from_numpy(albedo).cuda()
    tau = torch.empty((n, n, m), dtype=torch.float32, device="cuda")
    plan = nlos.Lct(n, m, w, dt)
    for _ in range(2):
        plan.forward(d_dev, a_dev, tau)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for a, b in ev:
        a.record()
        plan.forward(d_dev, a_dev, tau)
        b.record()
    torch.cuda.synchronize()
    lct_ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
    lct_tau = tau.cpu().numpy()
    plan.destroy()
    # the same surface through the direct sum
    pts = np.zeros((n * n, 8), np.float32)
    pts[:, 0], pts[:, 1], pts[:, 2] = X.ravel(), Y.ravel(), ((depth + 1) * cdt2).ravel()
    pts[:, 5], pts[:, 6], pts[:, 7] = -1.0, albedo.ravel(), (2 * w / n) ** 2
    prm = nlos.params(scan_nx=n, scan_ny=n, wall_half_x=w, wall_half_y=w, bin_width_s=dt,
                      num_bins=m, window_start_m=0.0, cos_mode="none")
    sc = nlos.scene_create(prm, torch.from_numpy(pts).cuda())
    dtau = torch.empty((n * n, m), dtype=torch.float32, device="cuda")
    for _ in range(2):
        nlos.forward(sc, dtau)
    torch.cuda.synchronize()
    for a, b in ev:
        a.record()
        nlos.forward(sc, dtau)
        b.record()
    torch.cuda.synchronize()
    direct_ms = float(np.median([a.elapsed_time(b) for a, b in ev]))
    d_tau = dtau.cpu().numpy().reshape(n, n, m).transpose(1, 0, 2)  # scan order is y-major
    sc.destroy()
    u, v = lct_tau.ravel().astype(np.float64), d_tau.ravel().astype(np.float64)
    corr = float(u @ v / (np.linalg.norm(u) * np.linalg.norm(v)))
    out = {"workload": "128 x 128 depth map (Gaussian bump on a tilted plane at 0.7-1.2 m), "
                       "1024 bins x 32 ps, 2 m wall, Beta(2,2) albedo",
           "grid": [2 * n, 2 * n, 2 * m], "lct_forward_ms": lct_ms,
           "direct_forward_ms": direct_ms, "direct_pairs": n * n * n * n,
           "shape_correlation_lct_vs_direct": corr}
    if peaks and peaks.get("dfma"):
        vol = (2 * n) * (2 * n) * (2 * m)
        flops = 2 * 5.0 * vol * math.log2(vol) + 6.0 * vol
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        peak = props.multi_processor_count * peaks["dfma"] * 2.0 * 2070e6
        achieved = flops / (lct_ms * 1e-3)
        out["lct_roofline"] = {
            "bound": "fp64", "achieved": achieved / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "peak_basis": f"{props.multi_processor_count} SMs x {peaks['dfma']:.2f} FP64 fma "
                          f"lanes/clk (measured) x 2 flops x 2070 MHz",
            "work_basis": "two 3-D radix-2 FFTs of the (2N)^2 (2M) volume, 5 V log2 V flops "
                          "each, and the spectral product (6 V)"}
    return out


def splat_moment_reds(params, pts, n_sample=128, seed=7):
    """Shared reductions per pass of the moment-form splat forward, counted on
    the host on a sample of scan points and scaled to the scan: six per
    (pair, bin window) whose moment row floor(u) - w0 + J lies inside the
    window's bw + 2J rows, for facing pairs of nonzero weight (the kernel's
    predicate). Windows as the launch chooses them: J = ceil(6 sigma) + 1,
    at most 256 - 2J bins each, rounded up to multiples of 4."""
    import math
    C = 299792458.0
    sig = params["jitter_fwhm_s"] / (2.0 * math.sqrt(2.0 * math.log(2.0)) * params["bin_width_s"])
    J = math.ceil(6.0 * sig) + 1
    B = params["num_bins"]
    max_bw = (256 - 2 * J) & ~3
    n_win = -(-B // max_bw)
    bw = ((-(-B // n_win)) + 3) & ~3
    nx, ny, w = params["scan_nx"], params["scan_ny"], params["wall_half_x"]
    rng = np.random.default_rng(seed)
    S = nx * ny
    ids = rng.choice(S, size=min(S, n_sample), replace=False)
    sx = -w + (ids % nx + 0.5) * (2 * w / nx)
    sy = -params["wall_half_y"] + (ids // nx + 0.5) * (2 * params["wall_half_y"] / ny)
    p = pts.astype(np.float64)
    q = p[:, 6] * p[:, 7]
    dx = sx[:, None] - p[None, :, 0]
    dy = sy[:, None] - p[None, :, 1]
    r = np.sqrt(dx * dx + dy * dy + p[None, :, 2] ** 2)
    cn = p[None, :, 3] * dx + p[None, :, 4] * dy - p[None, :, 5] * p[None, :, 2]
    j = np.floor(2.0 * r / (C * params["bin_width_s"]))  # no stand-off, L0 = 0
    ok = (cn > 0) & (q[None, :] > 0)
    count = 0
    for k in range(n_win):
        row = j - k * bw + J
        count += int(((row >= 0) & (row < bw + 2 * J) & ok).sum())
    return 6.0 * count * S / len(ids)


def splat_adjoint_bench(steps: int, warmup: int, peaks=None):
    """Differentiable path on the 8-scene glyph batch (64x64 scan, 65,536 points
    per scene, 512 bins x 8 ps, splat with 60 ps FWHM): per step, for every
    scene, the splat forward, the L2-loss gradient 2 (tau - target) and the
    hand-written adjoint (gradients for albedo and normal-offset depth)."""
    import torch
    import scenes
    from paper_2506_03747_gb300 import nlos
    params, sc_pts, tgt_pts = scenes.workload_glyph_batch()
    prm = nlos.params(params)
    stream = torch.cuda.current_stream()
    scs, targets, taus, gas, gds = [], [], [], [], []
    for pts, tp in zip(sc_pts, tgt_pts):
        sc = nlos.scene_create(prm, pts)
        tsc = nlos.scene_create(prm, tp)
        S, B, P = sc.num_scan, sc.num_bins, sc.num_points
        tgt = torch.empty((S, B), dtype=torch.float32, device="cuda")
        nlos.simulate(tsc, tgt)
        tsc.destroy()
        scs.append(sc)
        targets.append(tgt)
        taus.append(torch.empty((S, B), dtype=torch.float32, device="cuda"))
        gas.append(torch.empty(P, dtype=torch.float32, device="cuda"))
        gds.append(torch.empty(P, dtype=torch.float32, device="cuda"))
    S, B, P = scs[0].num_scan, scs[0].num_bins, scs[0].num_points
    g = torch.empty((S, B), dtype=torch.float32, device="cuda")
    fwd_ms, bwd_ms = [], []

    def step(record):
        for i, sc in enumerate(scs):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            e[0].record(stream)
            nlos.forward(sc, taus[i])
            e[1].record(stream)
            torch.sub(taus[i], targets[i], out=g)
            g.mul_(2.0)
            nlos.simulate_backward(sc, g, gas[i], gds[i])
            e[2].record(stream)
            if record:
                fwd_ms.append(e)
    for _ in range(warmup):
        step(False)
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        step(True)
    t1.record(stream)
    torch.cuda.synchronize()
    total = t0.elapsed_time(t1) * 1e-3
    f = sum(e[0].elapsed_time(e[1]) for e in fwd_ms) * 1e-3
    b = sum(e[1].elapsed_time(e[2]) for e in fwd_ms) * 1e-3
    pairs = len(scs) * S * P
    for sc in scs:
        sc.destroy()
    out = {"workload": "8 glyph-plane scenes, 64x64 scan, 65,536 points, 512 bins x 8 ps, "
                       "splat FWHM 60 ps, L2 loss",
           "pairs_per_step": pairs, "steps": steps,
           "ms_per_step": total * 1e3 / steps,
           "forward_pairs_per_s": steps * pairs / f,
           "adjoint_pairs_per_s": steps * pairs / b,
           "train_step_pairs_per_s": steps * pairs / total}
    # shared-atomic roofline of the splat forward (moment form: six shared
    # f32 reductions per pair and window in range)
    if peaks:
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        f_max = 2070e6
        reds = sum(splat_moment_reds(params, p) for p in sc_pts)
        achieved = steps * reds / f
        peak = props.multi_processor_count * peaks["red_f32"] * f_max
        out["forward_roofline"] = {
            "bound": "shared_atomic", "achieved": achieved / 1e9, "peak": peak / 1e9,
            "unit": "G red.shared.add.f32 lanes/s", "frac": achieved / peak,
            "peak_basis": f"{props.multi_processor_count} SMs x {peaks['red_f32']:.2f} lanes/clk "
                          f"(measured, all lanes active) x 2070 MHz",
            "work_basis": "6 reductions per (pair, bin window) with the moment row in range, "
                          "counted on the host on 128 sampled scan points per scene"}
        # FP32 roofline of the adjoint (moment form): every (scan point, point)
        # pair is evaluated, at ADJ_FP32_SLOTS_PER_PAIR FP32 issue slots each
        slots = ADJ_FP32_SLOTS_PER_PAIR[params.get("scan_mode", "confocal")]
        adj_peak = props.multi_processor_count * peaks["ffma"] * f_max / slots
        adj = steps * pairs / b
        out["adjoint_roofline"] = {
            "bound": "alu", "achieved": adj / 1e9, "peak": adj_peak / 1e9, "unit": "Gpair/s",
            "frac": adj / adj_peak,
            "peak_basis": f"{props.multi_processor_count} SMs x {peaks['ffma']:.1f} FMA lanes/clk "
                          f"(measured) x 2070 MHz / {slots} slots per pair "
                          f"({params.get('scan_mode', 'confocal')} scan)",
            "work_basis": "all S x P pairs (the adjoint culls none); its time includes the "
                          "moment-table kernel; 48 B per pair gathered from the L2-resident "
                          "moment tables"}
    return out


_POOLS = {}


def _serving_pools():
    """Point pools of the serving replays: one union scene and one heightfield
    of ~2M points; a request with P points takes the first P pool points (a
    view: no copy per request, so thousands of requests hold no more host
    memory than the pools; patch areas as in the pool)."""
    if not _POOLS:
        import scenes
        rng = np.random.default_rng(scenes.SEED_BASE + 55)
        pool_u, _ = scenes.primitive_union_points(rng, 2_000_000)
        pool_h = scenes.heightfield_points(rng, 1415)
        _POOLS["u"] = np.ascontiguousarray(pool_u[rng.permutation(len(pool_u))])
        _POOLS["h"] = np.ascontiguousarray(pool_h[rng.permutation(len(pool_h))])
    return _POOLS["u"], _POOLS["h"]


def serving_bench(n_requests: int, rate_hz: float, budget_gb: float = 120.0):
    """Replays one seeded Poisson-arrival trace (the serving workload: scan side
    16-256, bins 256-2048, 4-16 ps, 1e4-2e6 points, confocal or not, union or
    heightfield scene) through (i) the continuous-batching server and (ii) one
    request at a time (scene create + simulate + wait + destroy, in arrival
    order). Latency = result ready on the device (observed by the host) minus
    arrival."""
    import threading
    import torch
    import scenes
    from paper_2506_03747_gb300 import nlos

    reqs = scenes.serving_trace(n_requests=n_requests, rate_hz=rate_hz)
    pool_u, pool_h = _serving_pools()
    pts_of = []
    for r in reqs:
        pool = pool_u if r["kind"] == "union" else pool_h
        pts_of.append(pool[:min(r["n_points"], len(pool))])
    pairs = [r["params"]["scan_nx"] * r["params"]["scan_ny"] * len(p) for r, p in zip(reqs, pts_of)]

    # (i) continuous batching
    srv = nlos.server_create(int(budget_gb * (1 << 30)))
    t0 = time.perf_counter() + 0.05
    tickets = [None] * len(reqs)
    done_at = [None] * len(reqs)
    failures = []

    def submitter():
        for i, r in enumerate(reqs):
            dt = t0 + r["arrival_s"] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets[i] = srv.submit(r["params"], pts_of[i])

    th = threading.Thread(target=submitter)
    th.start()
    pending = set(range(len(reqs)))
    deadline = time.perf_counter() + 120.0 + reqs[-1]["arrival_s"]
    peak_resident, t_res = 0, 0.0
    while pending:
        if time.perf_counter() - t_res > 0.005:  # sampled, not on every poll: it takes the server lock
            peak_resident = max(peak_resident, srv.stats()["resident_bytes"])
            t_res = time.perf_counter()
        if time.perf_counter() > deadline:  # bounded: report what did not finish
            failures.append((sorted(pending)[:5], "not finished within the replay deadline"))
            for i in pending:
                done_at[i] = time.perf_counter()
            break
        for i in list(pending):
            if tickets[i] is None:
                continue
            try:
                st, _, _, _ = srv.poll(tickets[i], wait_ms=0)
            except nlos.NlosError as e:  # a failed request counts as done, reported
                failures.append((i, str(e)))
                st = nlos.OK
            if st == nlos.OK:
                done_at[i] = time.perf_counter()
                srv.release(tickets[i])
                pending.discard(i)
        time.sleep(0.0002)
    th.join()
    # SM cycles of the persistent kernel (posted when it exits, which it does
    # once the server parks it with nothing left to run)
    cyc, prev = None, None
    for _ in range(100):
        cyc = srv.device_cycles()
        if cyc == prev and sum(cyc.values()) > 0:
            break
        prev = cyc
        time.sleep(0.02)
    srv.destroy()
    lat_b = np.array([done_at[i] - (t0 + reqs[i]["arrival_s"]) for i in range(len(reqs))])
    span_b = max(done_at) - t0

    # (ii) one request at a time
    torch.cuda.synchronize()
    t0 = time.perf_counter() + 0.05
    done1 = []
    for i, r in enumerate(reqs):
        dt = t0 + r["arrival_s"] - time.perf_counter()
        if dt > 0:
            time.sleep(dt)
        prm = nlos.params(r["params"])
        sc = nlos.scene_create(prm, pts_of[i])
        S, B = sc.num_scan, sc.num_bins
        tau = torch.empty((S, B), dtype=torch.float32, device="cuda")
        cnt = torch.empty((S, B), dtype=torch.int32, device="cuda")
        nlos.simulate(sc, tau, cnt, None)
        torch.cuda.synchronize()
        done1.append(time.perf_counter())
        sc.destroy()
        del tau, cnt
    lat_1 = np.array([done1[i] - (t0 + reqs[i]["arrival_s"]) for i in range(len(reqs))])
    span_1 = max(done1) - t0
    tot_pairs = float(sum(pairs))

    def summ(lat, span):
        return {"p50_ms": float(np.percentile(lat, 50) * 1e3),
                "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "mean_ms": float(lat.mean() * 1e3),
                "req_per_s": len(lat) / span, "pairs_per_s": tot_pairs / span}

    return {"requests": len(reqs), "arrival_rate_hz": rate_hz, "budget_gb": budget_gb,
            "offered_pairs_per_s": tot_pairs / reqs[-1]["arrival_s"],
            "continuous_batching": dict(summ(lat_b, span_b), device_cycle_shares={
                k: v / max(1, sum(cyc.values())) for k, v in cyc.items()},
                peak_resident_bytes=int(peak_resident)),
            "one_at_a_time": summ(lat_1, span_1),
            "failures": failures[:5]}


def run_profile(args):
    """Runs `warmup` + `steps` bench steps of one workload (ingest + forward +
    detect), or forward passes only, and nothing else: the program that the
    ncu captures under profiles/ were taken of."""
    import torch
    from paper_2506_03747_gb300 import build as nbuild
    from paper_2506_03747_gb300 import nlos
    nbuild.build()
    if args.profile == "glyph":
        return _run_profile_glyph(args)
    params, pts_np = _workload(args.profile, 0)
    pts = torch.from_numpy(pts_np).cuda()
    sc = nlos.scene_create(nlos.params(params), pts)
    S, B = sc.num_scan, sc.num_bins
    tau = torch.empty((S, B), dtype=torch.float32, device="cuda")
    cnt = torch.empty((S, B), dtype=torch.int32, device="cuda")
    en = torch.empty(S, dtype=torch.float64, device="cuda")
    for _ in range(args.warmup + args.steps):
        if args.profile_forward:
            nlos.forward(sc, tau)
        else:
            nlos.scene_set_points(sc, pts)
            nlos.forward(sc, tau)
            nlos.detect(sc, tau, cnt, en)
    torch.cuda.synchronize()
    nlos.scene_check(sc)
    sc.destroy()
    return 0


def _run_profile_glyph(args):
    """Profile program of the differentiable path: one glyph scene of the
    8-scene batch (64x64 scan, 65,536 points, 512 bins x 8 ps, splat with 60 ps
    FWHM), each step the splat forward, the L2-loss gradient and the adjoint."""
    import torch
    import scenes
    from paper_2506_03747_gb300 import nlos
    params, sc_pts, tgt_pts = scenes.workload_glyph_batch(n_scenes=1)
    prm = nlos.params(params)
    sc = nlos.scene_create(prm, sc_pts[0])
    tsc = nlos.scene_create(prm, tgt_pts[0])
    S, B, P = sc.num_scan, sc.num_bins, sc.num_points
    target = torch.empty((S, B), dtype=torch.float32, device="cuda")
    nlos.simulate(tsc, target)
    tsc.destroy()
    tau = torch.empty_like(target)
    g = torch.empty_like(target)
    ga = torch.empty(P, dtype=torch.float32, device="cuda")
    gd = torch.empty(P, dtype=torch.float32, device="cuda")
    for _ in range(args.warmup + args.steps):
        nlos.forward(sc, tau)
        torch.sub(tau, target, out=g)
        g.mul_(2.0)
        nlos.simulate_backward(sc, g, ga, gd)
    torch.cuda.synchronize()
    nlos.scene_check(sc)
    sc.destroy()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle CPU baseline (profiling runs)")
    ap.add_argument("--cpu-scan", type=int, default=2048,
                    help="scan points in the CPU baseline sample")
    ap.add_argument("--ref-scan", type=int, default=256,
                    help="scan points per step of the reference (oracle) arm")
    ap.add_argument("--replicas", action="store_true",
                    help="with N > 1: every GPU simulates its own scene (weak scaling) instead "
                         "of one cube split by scan rows (strong scaling)")
    ap.add_argument("--union-steps", type=int, default=10,
                    help="timed steps of the union64 workload reported beside the headline "
                         "(0: skip)")
    ap.add_argument("--splat-steps", type=int, default=2,
                    help="steps of the differentiable-path measurement (0: skip)")
    ap.add_argument("--lct-steps", type=int, default=3,
                    help="timed passes of the FFT forward model comparison (0: skip)")
    ap.add_argument("--occlusion-steps", type=int, default=5,
                    help="timed forwards of the occlusion leg (0: skip)")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="requests in the serving replay (0: skip)")
    ap.add_argument("--serving-rate", type=float, default=200.0,
                    help="Poisson arrival rate of the serving replay [1/s]")
    ap.add_argument("--saturate-requests", type=int, default=400,
                    help="requests in the saturating serving leg (0: skip)")
    ap.add_argument("--saturate-rate", type=float, default=100000.0,
                    help="arrival rate of the saturating serving leg [1/s]")
    ap.add_argument("--profile", choices=["heightfield128", "union64", "glyph"], default=None,
                    help="only run warmup + steps bench steps of this workload (for ncu; "
                         "glyph: splat forward + adjoint of one configuration-4 scene)")
    ap.add_argument("--profile-forward", action="store_true",
                    help="with --profile: forward passes only")
    args = ap.parse_args()
    if args.profile:
        return run_profile(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
