#!/usr/bin/env python
"""Benchmark of one Levenberg-Marquardt iteration of photometric bundle
adjustment (damped solve: FP32 Cholesky with FP64 refinement in one
thread-block-cluster launch; box-plus update; linearisation of every pair at
the candidate; reduce, assemble, accept/reject) on one GB300.

Default workload: LiDAR spherical-projection BA, 50 frames of 64 x 1024
(vertical FOV -16.6..+16.6 deg) along a synthetic street, every pair with more
than 30% overlap, FP16 texels / FP32 residuals / FP64 solve.

Metric: residuals per second (valid pixel-point residuals linearised over
the timed iterations / their device time) and ms per iteration.  The timed
steps are consecutive iterations from the initial poses, after one untimed
linearisation and the warm-up iterations (the valid-residual count grows a
little as the poses converge); L2 is flushed (256 MiB write) before each step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the problem
on its own GPU (the path has no exchange step); value = all ranks' residuals /
the slowest rank's time.  --impl reference times the FP64 CPU oracle on the
host cores (rank 0 only).
"""
from __future__ import annotations

import argparse
import atexit
import json
import math
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "residuals/sec and ms per GN iteration, batched vs plain GPU path at stated error"
UNIT = "residuals/s"
WORKLOAD = ("lidar-street 50 frames 64x1024 spherical (vfov +-16.6 deg), pairs with >30% overlap, "
            "init noise 10 cm / 0.5 deg, 5% missing returns, FP16 texels / FP32 residuals / FP64-refined solve")
WORKLOADS = {"street": WORKLOAD,
             "room": ("rgbd-room 8 frames 160x120 pinhole (f 120), pairs j - i <= 3, init noise 2 cm / 1 deg, "
                      "FP16 texels / FP32 residuals / FP64-refined solve")}

# Algorithmic FP32 work of the linearisation kernel, counted from the formulas as
# implemented (FMA = 2 FLOP; square root, division and atan2 = 1):
# per processed point, transform 18 + spherical projection 13 = 31;
# per valid residual, taps and interpolation 51, residual / Huber / normal
# rotation 40, image gradients 118, d pi / d pbar 23, five Jacobian rows and
# their 6 x 6 accumulation 533 = 765.
FLOP_PER_POINT_SPHERICAL = 31
FLOP_PER_RESIDUAL_FULL = 765


def measured_hbm(path: str = None):
    """(GB/s, source): the HBM copy bandwidth measured on the GB300s
    (MEASURED_PEAKS.json), else the 6.8 TB/s fallback of one earlier GB300
    measurement."""
    path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured: MEASURED_PEAKS.json hbm_gbs"
    except (OSError, KeyError, ValueError, TypeError):
        return 6800.0, "fallback: 6.8 TB/s, one earlier GB300 measurement"


# dram__bytes_read.sum + dram__bytes_write.sum of one full k_linearize launch on this
# workload (ncu --set full capture of k_linearize<1, 1, 0, 3>, one launch after the autotuner's);
# to be retaken whenever the kernel changes
LINEARIZE_DRAM_BYTES = (370.882048 + 11.2384) * 1e6
# the same capture's unit utilisations (fraction of each unit's peak over the launch):
# SM issue, the L1 data pipe (the gathers), L2, DRAM
LINEARIZE_NCU_UNITS = {"sm_issue": 0.727, "l1_data_pipe": 0.575, "l2": 0.216, "dram": 0.041}
# normal estimation: neighbourhood radius clamp(NORMAL_SCALE / range, 1.5, NORMAL_MAX_RADIUS) pixels
NORMAL_SCALE = 8.0
NORMAL_MAX_RADIUS = 5
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1, help="GPUs of the run (N > 1 under torchrun: one replica per rank)")
    ap.add_argument("--steps", type=int, default=100, help="timed LM iterations")
    ap.add_argument("--warmup", type=int, default=3, help="untimed LM iterations before them")
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours",
                    help="ours: the GPU library; reference: the FP64 oracle on the host cores")
    ap.add_argument("--workload", choices=["street", "room"], default="street",
                    help="street: 50 LiDAR frames of 64 x 1024 (the benchmark); room: 8 RGB-D frames of 160 x 120")
    ap.add_argument("--no-plain", action="store_true", help="skip timing the plain per-pair path")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end run from pinned host buffers")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="CPU oracle sample budget")
    return ap.parse_args()


def make_workload(name):
    from paper_2303_16878_gb300 import synth
    if name == "room":
        return synth.make_rgbd_room()
    if name == "street":
        return synth.make_lidar_street()
    raise ValueError(f"unknown workload {name!r}")


# ----------------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons.  Started before the
    warm-up so that short timed regions still see samples: mark() brackets the
    timed region, and stop() keeps the samples taken inside it (widened by
    `slack` seconds on both sides when it holds fewer than three)."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, interval_ms: int = 20):
        self.proc = None
        self.path = None
        self.gpu = gpu_index
        self.window = None
        if shutil.which("nvidia-smi"):
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", str(interval_ms)],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            atexit.register(self._end)  # never outlive the bench, whatever ends it

    def _end(self):
        if self.proc and self.proc.poll() is None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def wait_first(self, timeout_s: float = 10.0) -> bool:
        """Block until nvidia-smi has written its first row (it takes a moment to
        start), at most timeout_s; True when a row is there."""
        if not self.proc:
            return False
        deadline = time.time() + timeout_s
        while time.time() < deadline:
            if os.path.getsize(self.path) > 0:
                return True
            if self.proc.poll() is not None:
                return False
            time.sleep(0.05)
        return False

    def mark(self, t0: float, t1: float):
        """The timed region, as time.time() values."""
        self.window = (t0, t1)

    def stop(self, slack: float = 0.5):
        if not self.proc:
            return None
        self._end()
        with open(self.path) as fh:
            rows = parse_clock_lines(fh)
        os.unlink(self.path)
        return summarise_clocks(rows, self.window, slack)


def parse_clock_lines(lines):
    """Rows of the ClockSampler query (nvidia-smi csv, noheader, nounits)."""
    from datetime import datetime
    rows = []
    for line in lines:
        f = [x.strip() for x in line.split(",")]
        if len(f) < 10:
            continue
        try:
            ts = datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            rows.append(dict(ts=ts, sm=float(f[2]), max=float(f[3]),
                             power=float(f[4]) if f[4] not in ("[N/A]", "") else 0.0,
                             hw=f[6], hw_th=f[7], sw_th=f[8], pcap=f[9]))
        except ValueError:
            continue
    return rows


def summarise_clocks(rows, window=None, slack: float = 0.5):
    """Median SM clock under load, the max clock and the throttle reasons seen
    within the window (t0, t1) (widened by slack seconds when it holds fewer
    than three samples)."""
    in_region = rows
    widened = False
    if window is not None:
        t0, t1 = window
        in_region = [r for r in rows if t0 <= r["ts"] <= t1]
        if len(in_region) < 3:
            in_region = [r for r in rows if t0 - slack <= r["ts"] <= t1 + slack]
            widened = True
    if not in_region:
        return None
    reasons = set()
    for r in in_region:
        for key, name in (("hw", "hw_slowdown"), ("hw_th", "hw_thermal_slowdown"),
                          ("sw_th", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
            if r[key].lower().startswith("active"):
                reasons.add(name)
    top = max(x["power"] for x in in_region)
    loaded = [r["sm"] for r in in_region if r["power"] > 0.25 * top] or [r["sm"] for r in in_region]
    return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r["max"] for r in in_region),
            "reasons": sorted(reasons), "samples": len(in_region),
            "window": "timed region +- %.1f s" % slack if widened else "timed region"}


# ----------------------------------------------------------------------------- ranks

def reduce_over_ranks(seconds_or_ms: float, units: float, world: int, device=None):
    """Whole-job aggregation across ranks: the slowest rank's time and the sum
    of every rank's units (residuals).  With world == 1 the inputs pass through."""
    if world <= 1:
        return float(seconds_or_ms), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds_or_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ----------------------------------------------------------------------------- GPU arm

def run_ours(args, rank, world, device):
    import torch
    import paper_2303_16878_gb300 as pba

    # clock sampling starts before the set-up, so that nvidia-smi is emitting
    # rows well before the timed region
    clocks = ClockSampler(device.index if device.index is not None else 0)
    w = make_workload(args.workload)
    # a dedicated stream: the library enqueues on it and the events below are recorded on it
    stream = torch.cuda.Stream(device)
    torch.cuda.set_stream(stream)
    prob = pba.problem_from_workload(w, path=pba.PBA_PATH_BATCHED, texel=pba.PBA_TEXEL_F16, stream=stream,
                                     solver=pba.PBA_SOLVE_MIXED)
    init = np.ascontiguousarray(w.poses_init.reshape(-1, 12))
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=device)
    n_points_total = sum(prob.frame_points(int(i)) for i, _ in w.pairs)

    def start(p):
        # every run starts from the initial poses with automatic damping; the
        # first linearisation is not part of any timed iteration
        p.set_poses(init)
        p.set_lambda(None)
        p.linearize()

    def one_step(p):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p.iterate_async(1)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), p.get_stats()

    variants = prob.autotune(2)
    clocks.wait_first()
    start(prob)
    for _ in range(args.warmup):
        one_step(prob)
    launches = prob.iteration_launches()

    # timed region: K consecutive iterations
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    epoch0 = time.time()
    wall0 = time.perf_counter()
    ms, nvalid, stats = [], [], None
    for _ in range(args.steps):
        t, stats = one_step(prob)
        ms.append(t)
        nvalid.append(stats["n_valid"])
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clocks.mark(epoch0, time.time())
    clk = clocks.stop()
    if world > 1:
        torch.distributed.barrier()
    total_ms, res_all = reduce_over_ranks(float(sum(ms)), float(sum(nvalid)), world, device)
    value = res_all / (total_ms / 1e3)
    ms_per_step = total_ms / args.steps

    # per-phase device times (same stream, same flush), for the roofline
    phases = {}
    start(prob)
    for _ in range(args.steps):
        flush.zero_()
        _, ph = prob.iterate_timed()
        for k, v in ph.items():
            phases.setdefault(k, []).append(v)
    phase_ms = {k: float(np.mean(v)) for k, v in phases.items()}

    out = dict(value=value, ms_per_step=ms_per_step, n_valid=int(nvalid[-1]), n_valid_mean=float(np.mean(nvalid)),
               launches=launches, clocks=clk,
               phase_ms=phase_ms, wall_s=wall, n_points=int(n_points_total), n_pairs=int(len(w.pairs)),
               stats=stats, variants=variants)

    # adjoint of the total cost (pose / extrinsic / image gradients), events on the same stream
    start(prob)
    adj = {}
    for images in (False, True):
        ts = []
        for _ in range(3):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            prob.cost_gradient(poses=True, extrinsics=True, images=images, device=device)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1))
        adj["with_image_gradient_ms" if images else "poses_extrinsic_ms"] = float(np.median(ts))
    out["adjoint"] = adj

    # graph construction (Sec. IV-B) over every same-sensor candidate within 30 deg / 40 m
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    gp, _ = prob.build_pairs(math.radians(30.0), 40.0, 0.3, True)
    out["build_pairs"] = {"ms": 1e3 * (time.perf_counter() - t0), "pairs_kept": int(len(gp)),
                          "criteria": "angle < 30 deg, translation < 40 m, valid ratio > 0.3, sequential edges"}

    # normal estimation (Sec. IV-A) of every frame from its depth, then the rebuild of
    # texels and pixel-points; the problem's later use (e2e) uploads the frames again
    nts, nwall = [], []
    for _ in range(3):
        flush.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record(stream)
        prob.estimate_normals(0, w.n_frames, scale=NORMAL_SCALE, max_radius=NORMAL_MAX_RADIUS)
        e1.record(stream)
        e1.synchronize()
        nwall.append(1e3 * (time.perf_counter() - t0))
        nts.append(e0.elapsed_time(e1))
    out["normals"] = {"device_ms": float(np.median(nts)), "call_ms": float(np.median(nwall)),
                      "frames": int(w.n_frames), "scale": NORMAL_SCALE, "max_radius": NORMAL_MAX_RADIUS,
                      "points_after": int(sum(prob.frame_points(k) for k in range(w.n_frames)))}

    # the same iteration with the FP64 Cholesky solver (phase times only)
    f64 = pba.problem_from_workload(w, path=pba.PBA_PATH_BATCHED, texel=pba.PBA_TEXEL_F16, stream=stream,
                                    solver=pba.PBA_SOLVE_CHOLESKY_F64)
    f64.autotune(1)
    f64_solve = []
    start(f64)
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        _, ph = f64.iterate_timed()
        f64_solve.append(ph["solve"])
    f64.close()
    out["solve_update_f64_ms"] = float(np.mean(f64_solve))

    # plain per-pair path on the same workload
    if not args.no_plain:
        plain = pba.problem_from_workload(w, path=pba.PBA_PATH_PLAIN, texel=pba.PBA_TEXEL_F32, stream=stream,
                                          solver=pba.PBA_SOLVE_MIXED)
        start(plain)
        for _ in range(max(1, args.warmup)):
            one_step(plain)
        pms = []
        for _ in range(max(3, args.steps // 2)):
            t, _ = one_step(plain)
            pms.append(t)
        plain.close()
        out["plain_ms_per_step"] = float(np.mean(pms))

    # end to end through the C ABI from pinned host buffers
    if not args.no_e2e:
        chans = torch.from_numpy(w.channels_array()).pin_memory()
        poses_h = torch.from_numpy(init.copy()).pin_memory()
        out_h = torch.empty_like(poses_h).pin_memory()
        h2d = chans.numel() * 4 + poses_h.numel() * 8
        d2h = out_h.numel() * 8 + 48
        walls, ev = [], 0
        for k in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            prob.upload_frames(0, chans)
            prob.set_poses(poses_h)
            prob.set_lambda(None)
            prob.iterate_async(1)
            st = prob.get_stats()
            prob._check(prob._lib.pba_get_poses(prob._h, out_h.data_ptr()), "get_poses")
            t1 = time.perf_counter()
            if k >= args.warmup:
                walls.append(t1 - t0)
                ev += st["n_valid"]
        wall_max, ev_all = reduce_over_ranks(sum(walls), float(ev), world, device)
        e2e_local = ev_all / wall_max
        out["e2e"] = {"value": e2e_local, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                      "ms_per_step": 1e3 * sum(walls) / len(walls)}
    prob.close()
    return out, w


# ----------------------------------------------------------------------------- CPU oracle

def oracle_sample(w, seconds, seed=0, part=(0, 1)):
    """Time the FP64 oracle's LM iteration work (full linearisation + cost
    re-evaluation) on a seeded sample of pairs of the same workload, one core.
    part = (k, n): only every n-th pair of the seeded order from the k-th on
    (the slice of worker k of n)."""
    import oracle
    oracle.build()
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(w.pairs))[part[0]::part[1]]
    s = w.sensors[0]
    done_res, elapsed, used = 0, 0.0, 0
    for q in order:
        i, j = w.pairs[q]
        t0 = time.perf_counter()
        r = oracle.linearize_pair(s, w.params, w.channels[i], w.channels[j], w.poses_init[i], w.poses_init[j])
        oracle.linearize(w.sensors, w.frame_sensor, w.channels, w.poses_init, w.pairs[q:q + 1], w.params,
                         want_system=False)
        elapsed += time.perf_counter() - t0
        done_res += r["count"]
        used += 1
        if elapsed >= seconds:
            break
    return dict(value=done_res / elapsed, unit=UNIT, cores=1, kind="oracle",
                sample=f"{used} of {len(w.pairs)} pairs (seeded), full linearisation + cost re-evaluation, "
                       f"{done_res} residuals in {elapsed:.1f} s, single-threaded FP64 C",
                seconds=elapsed, pairs=used, residuals=done_res)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def _oracle_worker(workload_name, k, n, inbox, outbox):
    """Worker k of n: builds the workload once, then times its slice of the
    seeded pair order for every (seconds, seed) it receives (None ends it)."""
    w = make_workload(workload_name)
    import oracle
    oracle.build()
    outbox.put(("ready", k))
    while True:
        task = inbox.get()
        if task is None:
            return
        seconds, seed = task
        outbox.put(oracle_sample(w, seconds, seed=seed, part=(k, n)))


class OraclePool:
    """The oracle on every host core: n processes started with spawn (safe after
    CUDA initialisation), each holding the workload.  A sample sends the same
    (seconds, seed) to all of them at once; they time disjoint slices of one
    seeded pair order concurrently, and the rate is all residuals over the
    slowest worker's time."""

    def __init__(self, workload_name: str, workers: int = None, ready_timeout: float = 300.0):
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        self.n = workers or host_cores()
        self.outbox = ctx.Queue()
        self.inboxes = [ctx.Queue() for _ in range(self.n)]
        self.procs = [ctx.Process(target=_oracle_worker, args=(workload_name, k, self.n, self.inboxes[k], self.outbox),
                                  daemon=True) for k in range(self.n)]
        for pr in self.procs:
            pr.start()
        try:
            self._collect(ready_timeout)
        except Exception:
            self.close()
            raise

    def _collect(self, timeout: float) -> list:
        """One message from every worker; raises as soon as a worker has died,
        or after timeout seconds."""
        import queue
        out, deadline = [], time.time() + timeout
        while len(out) < self.n:
            try:
                out.append(self.outbox.get(timeout=1.0))
            except queue.Empty:
                dead = [pr.exitcode for pr in self.procs if pr.exitcode is not None]
                if dead:
                    raise RuntimeError(f"oracle worker exited with code {dead[0]}")
                if time.time() > deadline:
                    raise TimeoutError(f"oracle workers: {len(out)} of {self.n} answered in {timeout:.0f} s")
        return out

    def sample(self, seconds: float, seed: int = 0) -> dict:
        for q in self.inboxes:
            q.put((seconds, seed))
        rs = self._collect(3 * seconds + 120)
        res = sum(r["residuals"] for r in rs)
        elapsed = max(r["seconds"] for r in rs)
        pairs = sum(r["pairs"] for r in rs)
        return dict(value=res / elapsed, unit=UNIT, cores=self.n, kind="oracle",
                    sample=f"{pairs} pairs (seeded, split over {self.n} processes), full linearisation + cost "
                           f"re-evaluation, {res} residuals in {elapsed:.1f} s, FP64 C, one process per host core",
                    seconds=elapsed, pairs=pairs, residuals=res)

    def close(self):
        for q in self.inboxes:
            try:
                q.put(None)
            except Exception:
                pass
        for pr in self.procs:
            pr.join(timeout=10)
            if pr.is_alive():
                pr.terminate()


def run_reference(args):
    per_step = max(0.5, min(args.cpu_seconds, 150.0 / max(1, args.steps + args.warmup)))
    pool = OraclePool(args.workload)
    cores = pool.n
    vals, secs = [], []
    try:
        for k in range(args.warmup + args.steps):
            r = pool.sample(per_step, seed=k)
            if k >= args.warmup:
                vals.append(r["value"])
                secs.append(r["seconds"])
    finally:
        pool.close()
    value = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: seeded pairs of the workload split over {cores} processes "
                                       f"(one per host core), each process timing at most {per_step:.1f} s of "
                                       f"FP64 oracle work (full + cost linearisation) or its whole slice"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# ----------------------------------------------------------------------------- the JSON line

def make_line(args, world: int, out: dict, n_frames: int, n_sms: int, hbm_peak_gbs: float,
              hbm_source: str = "measured: MEASURED_PEAKS.json hbm_gbs") -> dict:
    """The GPU arm's JSON line from the measurements in `out` (pure: no device
    access).  Roofline of the dominant kernel: algorithmic FP32 FLOPs of one
    full linearisation (per valid residual and per processed point, mean
    valid count of the timed iterations) over its CUDA-event duration, against
    the nominal FP32 ALU peak at the sampled maximum SM clock."""
    ph = out["phase_ms"]
    lin_ms = ph["linearize"]
    n_valid = out.get("n_valid_mean", out["n_valid"])
    flops = n_valid * FLOP_PER_RESIDUAL_FULL + out["n_points"] * FLOP_PER_POINT_SPHERICAL
    sm_max = (out["clocks"] or {}).get("sm_max_mhz") or 2070.0
    peak = n_sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = flops / (lin_ms / 1e3) / 1e12
    line = {
        "metric": METRIC, "value": out["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": out["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[getattr(args, "workload", "street")], "frames": n_frames,
                   "pairs": out["n_pairs"],
                   "points_per_iteration": out["n_points"], "residuals_per_iteration": n_valid,
                   "l2": "flushed before every timed step (256 MiB write)",
                   "steps": "consecutive LM iterations from the initial poses (one untimed linearisation first)",
                   "parallelism": f"replicas x{world}", "autotuned_variants": list(out["variants"])},
        # each residual is a 5-vector (g, d, n_x, n_y, n_z)
        "scalar_residuals_per_s": 5.0 * out["value"],
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": LINEARIZE_DRAM_BYTES, "kernel": "k_linearize<f16, full>",
                     "kernel_ms": lin_ms, "peak_source": "nominal: SMs x 128 FP32 lanes x 2 x max SM clock",
                     "hbm": {"traffic_bytes": LINEARIZE_DRAM_BYTES, "peak_gbs": hbm_peak_gbs,
                             "frac": LINEARIZE_DRAM_BYTES / (lin_ms / 1e3) / 1e9 / hbm_peak_gbs,
                             "peak_source": hbm_source},
                     "ncu_unit_fracs": LINEARIZE_NCU_UNITS,
                     "binding": "SM instruction issue, then the L1 data pipe of the gathers"},
        "phase_ms": ph,
        "solver": "FP32 Jacobi-scaled Cholesky + FP64 iterative refinement (|r| <= 1e-10 |b|), one thread-block-cluster launch",
        "solve_f64_cholesky_ms": out["solve_update_f64_ms"],
        "lm_step": "speculative: linearise in full at the candidate; its system becomes current on acceptance",
        "gpu_launches": out["launches"] * args.steps,
        "clocks": out["clocks"],
    }
    for k in ("build_pairs", "normals", "adjoint", "e2e"):
        if k in out:
            line[k] = out[k]
    if "plain_ms_per_step" in out:
        line["plain_ms_per_step"] = out["plain_ms_per_step"]
        line["speedup_vs_plain"] = out["plain_ms_per_step"] / out["ms_per_step"]
    return line


# ----------------------------------------------------------------------------- main

def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    import torch
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (the GPU path has no CPU fallback)")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=device)
    out, w = run_ours(args, rank, world, device)
    if rank == 0:
        sms = torch.cuda.get_device_properties(device).multi_processor_count
        line = make_line(args, world, out, w.n_frames, sms, *measured_hbm())
        if not args.no_cpu and world == 1:
            one = oracle_sample(w, args.cpu_seconds)
            try:
                pool = OraclePool(args.workload)
                try:
                    cb = pool.sample(args.cpu_seconds)
                finally:
                    pool.close()
            except Exception as e:  # the single-process figure still stands
                cb = dict(one, sample=one["sample"] + f" (parallel run failed: {type(e).__name__})")
            line["cpu_baseline"] = {k: cb[k] for k in ("value", "unit", "cores", "kind", "sample")}
            line["cpu_baseline_one_core"] = {k: one[k] for k in ("value", "unit", "cores", "kind", "sample")}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
