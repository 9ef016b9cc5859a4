"""Benchmark: rays/s of one whole magnification-map step on GB300.

A step is one pass of the whole path over one synthetic paper-scale field
(13,000 lognormal lenses, kappa = 0.48, gamma = 0.50, kappa_* = 0.005, 1e11
rays, 8192^2 uint32 map): field set-up (parameters, lens binning, Taylor
order, far-field coefficients at every level-2 node), shooting all rays,
the magnification map (Eq. 12) and ten Gaussian-source light curves.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `value` is measured with inputs resident in
device memory; `e2e` repeats the step through the C ABI with host buffers
(lens upload and the map's device-to-host read inside the timed region).
The reference arm (--impl reference) times the FP64 CPU oracle on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import signal
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rays/s at 13k lenses on 1 GB300; % FP32 peak; map L1 err vs FP64 oracle"
UNIT = "rays/s"
N_TRACKS, TRACK_SAMPLES, SIGMA_PX = 10, 4096, 0.5
# FP32 FMA units of GB300 (152 SMs x 128 lanes) at the maximum SM clock: the
# derived peak, reported beside the measured one (ml_fp32_fma_peak)
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
# copy bandwidth of the GB300s (GB/s), the HBM roofline's denominator
HBM_GBS_FALLBACK = 6790.0
# DRAM bytes per ray of the certified counting kernel, from one ncu capture
# per workload (dram__bytes_read.sum + dram__bytes_write.sum of one launch
# over a centred slice of the lattice at the autotuned grid: 2e10 rays of the
# paper-scale map, 2e9 of the Table-1 fold field, whose 84 MB map stays in
# L2), valid for the kernel sources whose code (comments and blank space left
# out, code_hash) has these sha1 prefixes only.
TRAFFIC_BYTES_PER_RAY = {"paper": (216.402944e6 + 269.967104e6) / 2.0e10,
                         "fold": (23.782144e6 + 512.0) / 2.0e9}
TRAFFIC_SOURCES = {"ml_shoot.cu": "48c686ae", "ml_internal.cuh": "4806c1e0", "ml_task.cuh": "3d1d5136"}


def code_hash(text: str) -> str:
    """sha1 of a C++/CUDA source's code: comments, blank lines and spacing
    left out, so that editing a comment does not count as a kernel change."""
    import hashlib
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    lines = (" ".join(re.sub(r"//.*$", "", ln).split()) for ln in text.splitlines())
    return hashlib.sha1("\n".join(ln for ln in lines if ln).encode()).hexdigest()


# The library's kernels in one field build: k_lens_cells, k_scan, k_scatter,
# k_p_bound, k_lens_l1, k_outer_csr, k_box_p2l, k_sub_p2l, k_node_shift,
# k_node_finalize.  A step adds the shooting launches, mu and the light curves
# (the fold step: the two peak kernels; the differentiable step: the CIC
# forward, mu, and k_adj_rays, k_adj_far, k_adj_unsort).
BUILD_KERNELS = 10
# distance bins of the fold step's peak statistics: beta_x from 0.02 to 63 theta_E,
# four per decade (the fold map spans beta_x in [0, 40])
FOLD_DISTANCE_EDGES = [0.02 * 10.0 ** (k / 4.0) for k in range(15)]


def fold_peak_summary(stats, info):
    """Per distance bin: true peaks, crossings per theta_E of curve and the
    mean peak magnification (Figs. 4-5, before the paper's normalisations)."""
    n, s, pos = (np.asarray(a, np.float64) for a in stats)
    with np.errstate(divide="ignore", invalid="ignore"):
        dens = np.where(pos > 0, n / (pos * info["dpx"]), 0.0)
        mu = np.where(n > 0, s * info["mu_per_count"] / n, 0.0)
    return {"edges_theta_e": [round(e, 4) for e in FOLD_DISTANCE_EDGES],
            "n_peaks": [int(v) for v in stats[0]],
            "crossings_per_theta_e": [round(float(v), 4) for v in dens],
            "mean_mu_peak": [round(float(v), 3) for v in mu]}


def traffic_per_launch(rays_per_launch: float, workload: str = "paper", walk: str = "certified"):
    """Measured DRAM bytes per launch of a workload's certified walk, or None
    for another kernel or once the kernel has changed."""
    if walk != "certified" or workload not in TRAFFIC_BYTES_PER_RAY:
        return None
    csrc = os.path.join(ROOT, "paper_2308_14278_gb300", "csrc")
    for name, prefix in TRAFFIC_SOURCES.items():
        with open(os.path.join(csrc, name)) as fh:
            if not code_hash(fh.read()).startswith(prefix):
                return None
    return TRAFFIC_BYTES_PER_RAY[workload] * rays_per_launch


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="paper", choices=["paper", "fold", "batched", "differentiable"],
                    help="paper: one 1e11-ray map (the headline line); batched: 80 maps in one "
                         "graph-captured persistent launch against the same maps one at a time; "
                         "differentiable: CIC forward + adjoint of 1,000 lenses and 4e8 rays; "
                         "fold: the Table-1 fold field (13,745 lenses, 2048x10240 map)")
    ap.add_argument("--rays", type=float, default=1e11)
    ap.add_argument("--map-px", type=int, default=8192)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--clocks-dir", default=None,
                    help="directory for the nvidia-smi clock samples of the timed region "
                         "(default: a temporary directory); the JSON line carries their summary")
    ap.add_argument("--independent", action="store_true",
                    help="N > 1: one independent map per rank (weak scaling) instead of ONE "
                         "paper-scale map shot across the ranks (contiguous level-1 bands per "
                         "rank, integer map sum onto rank 0 over NCCL; strong scaling, the "
                         "default); with --workload batched, each rank runs its own 80 maps "
                         "instead of splitting one set (whole maps balanced by rays)")
    ap.add_argument("--no-independent", action="store_true",
                    help="N > 1: skip the weak-scaling companion record of a sharded run")
    ap.add_argument("--fp32-peak-only", action="store_true",
                    help="print the measured FP32 FMA peak (ml_fp32_fma_peak) as JSON and exit")
    ap.add_argument("--no-sub", action="store_true",
                    help="skip the batched and differentiable sub-records of the default line")
    ap.add_argument("--no-tune", action="store_true",
                    help="the paper's level-2 grid (L2 = L1/20) instead of the autotuned one")
    ap.add_argument("--grid", default="",
                    help="profiling: fix the grid the autotuner chose, 'L1X,L1Y,SX,SY[,FAR]' "
                         "(level-1 cell size in theta_E, level-2 subdivisions and, optionally, "
                         "the certified walk's lens distance in lattice spacings, 'inf' for "
                         "lens columns walked per ray), instead of tuning again")
    ap.add_argument("--walk", default="certified", choices=["certified", "per_ray"],
                    help="ray walk of the counting kernel: certified spans (default) or every "
                         "ray evaluated; both give bit-identical maps")
    ap.add_argument("--shoot-rays", type=float, default=0,
                    help="profiling: shoot only this many rays (a centred slice of the lattice) "
                         "per step; the default shoots them all")
    return ap.parse_args()


def grid_kwargs(args, w):
    """Field keyword arguments for the grid: the autotuner's (default), the
    paper's (--no-tune) or a fixed one (--grid, which sets w.l1)."""
    import paper_2308_14278_gb300 as ml
    walk = ml.WALK_PER_RAY if getattr(args, "walk", "certified") == "per_ray" else ml.WALK_CERTIFIED
    if not args.grid:
        return dict(tune=not args.no_tune, walk=walk)
    vals = args.grid.split(",")
    l1x, l1y, sx, sy = (float(v) for v in vals[:4])
    w.l1 = (l1x, l1y)
    kw = dict(tune=False, l2_sub=(int(sx), int(sy)), walk=walk)
    if len(vals) > 4:
        kw["span_far"] = 3.0e38 if vals[4].strip() == "inf" else float(vals[4])
    return kw


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi samples of the SM clock, power and throttle reasons every
    50 ms while the block runs.  Entering waits for the first sample, so that
    sampling is under way when the timed region starts; summary() keeps the
    samples taken between entry and exit (by their timestamps)."""
    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 50

    def __init__(self, index: int, directory: str | None = None, tag: str = ""):
        self.index = index
        self.proc = None
        self.t_in = self.t_out = None
        d = directory or os.path.join(tempfile.gettempdir(), f"ml_bench_clocks_{os.getpid()}")
        self.path = os.path.join(d, f"clocks{tag}_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}",
                                          f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", str(self.PERIOD_MS)], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
            deadline = time.time() + 5.0
            while time.time() < deadline and self.proc.poll() is None:
                with open(self.path) as fh:
                    if fh.read().count("\n") >= 1:
                        break
                time.sleep(0.02)
        except Exception:
            self.proc = None
        self.t_in = time.time()
        return self

    def __exit__(self, *exc):
        self.t_out = time.time()
        if self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    @staticmethod
    def _epoch(stamp: str):
        import datetime
        try:
            return datetime.datetime.strptime(stamp.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        rows = []
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                sm, mx = float(parts[2]), float(parts[3])
            except ValueError:
                continue
            rows.append((self._epoch(parts[0]), sm, mx,
                         {nm for nm, v in zip(names, parts[6:10]) if v.lower() == "active"}))
        if not rows:
            return None
        pad = self.PERIOD_MS / 1e3
        inside = [r for r in rows if r[0] is not None and self.t_in is not None and
                  self.t_in - pad <= r[0] <= self.t_out + pad]
        use = inside or rows
        sm = [r[1] for r in use]
        load = [v for v in sm if v > 0.5 * max(sm)] or sm
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": float(max(r[2] for r in use)),
                "reasons": sorted(set().union(*(r[3] for r in use))), "samples": len(use),
                "period_ms": self.PERIOD_MS, "in_timed_region": bool(inside)}


# ---------------------------------------------------------------------------
# measured FP32 peak
# ---------------------------------------------------------------------------

PEAK_ITERS = 1 << 21


def measure_fp32_peak(ml, torch, stream, local, clocks_dir=None, launches=5):
    """FP32 FMA throughput of this GPU measured by the library's probe
    (ml_fp32_fma_peak: 4 blocks of 256 threads per SM, eight independent FMA
    chains per thread), best of `launches` CUDA-event-timed launches for
    scalar FFMA and for the two-lane fma.rn.f32x2, with the SM clock sampled
    meanwhile.  TFLOP/s, 2 flop per FMA."""
    sink = torch.zeros(8 * 1024, dtype=torch.float32, device=f"cuda:{local}")
    out = {}
    with ClockSampler(local, clocks_dir, tag="_fp32peak") as clk:
        for two in (False, True):
            ml.ml_fp32_fma_peak(two, 4, 1 << 12, sink, stream)        # warm-up
            best = 0.0
            for _ in range(launches):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                flop = ml.ml_fp32_fma_peak(two, 4, PEAK_ITERS, sink, stream)
                e1.record(stream)
                e1.synchronize()
                best = max(best, flop / (e0.elapsed_time(e1) / 1e3) / 1e12)
            out["two_lane_tflops" if two else "scalar_tflops"] = best
        torch.cuda.synchronize()
    c = clk.summary()
    if c:
        out["sm_mhz"] = c["sm_mhz"]
        out["reasons"] = c["reasons"]
    out["derived_tflops_at_max_clock"] = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    return out


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------

def hbm_peak_gbs():
    """Measured copy bandwidth of this machine's GPUs (generated file),
    else the recorded fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured (MEASURED_PEAKS.json)"
    except Exception:
        return HBM_GBS_FALLBACK, "fallback"


def run_ours(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    import paper_2308_14278_gb300 as ml
    from paper_2308_14278_gb300 import inputs, shard
    ml.load()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # N > 1: one map shared by the ranks, each shooting its part of the lattice
    # and the integer maps summed onto rank 0 (strong scaling, the design's
    # exchange step); --independent: one map of its own per rank (weak)
    sharded = world > 1 and not args.independent
    seed = 0 if sharded else rank
    if args.workload == "fold":
        w = inputs.fold_field(seed=seed, n_rays=args.rays, n_tracks=N_TRACKS)
    else:
        w = inputs.paper_map(seed=seed, n_rays=args.rays, map_px=args.map_px, n_tracks=N_TRACKS)
    grid_kw = grid_kwargs(args, w)
    counts_buf = (torch.empty((w.map_n[1], w.map_n[0]), dtype=torch.int32, device=f"cuda:{local}")
                  if sharded else None)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    lens_dev = [torch.from_numpy(a).to(dev) for a in (w.lenses.x, w.lenses.y, w.lenses.m)]
    tracks = inputs.tracks(N_TRACKS, w.map_n[0], w.map_n[1], 4 * SIGMA_PX + 1, seed=100 + rank)
    mu_out = torch.empty((w.map_n[1], w.map_n[0]), dtype=torch.float32, device=dev)
    lc_out = torch.empty((N_TRACKS, TRACK_SAMPLES), dtype=torch.float32, device=dev)
    peak_mask = (torch.empty(w.map_n[0] * w.map_n[1] + 4, dtype=torch.uint8, device=dev)
                 if args.workload == "fold" else None)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > L2 (129 MB)
    # the map is consumed (mu, light curves, peaks) where it is whole: on every
    # rank of independent maps, on rank 0 of a sharded one
    consumer = (not sharded) or rank == 0

    def make_desc(device_lenses: bool, host_lenses=None):
        d = ml.make_desc(w, precision=ml.PREC_MIXED, lens_arrays=host_lenses, **grid_kw)
        if device_lenses:
            d.lens_x, d.lens_y, d.lens_m = (t.data_ptr() for t in lens_dev)
            d.lens_mem_is_device = 1
        return d

    ev = lambda: torch.cuda.Event(enable_timing=True)   # noqa: E731
    info_holder = {}

    def step(timers=None):
        e = [ev() for _ in range(5)] if timers is not None else None
        if e: e[0].record(stream)
        h = ml.ml_field_create(make_desc(True), stream)
        info = ml.ml_field_info(h)
        if e: e[1].record(stream)
        n_all = info["n_rays_x"] * info["n_rays_y"]
        n_shoot = int(min(args.shoot_rays, n_all)) if args.shoot_rays else n_all
        r0 = (n_all - n_shoot) // 2
        if sharded:
            a, b = shard.ray_ranges(info["n_rays_x"], info["n_rays_y"], info["n1y"], world)[rank]
            ml.ml_shoot_rays(h, a, b, stream)
            ml.ml_magnification_map(h, ml.MAP_COUNTS_U32, counts_buf, stream)
            shard.reduce_counts(counts_buf, dst=0)   # NCCL integer sum onto rank 0
            if consumer:
                ml.ml_field_set_counts(h, counts_buf, stream)
        else:
            ml.ml_shoot_rays(h, r0, r0 + n_shoot, stream)
        if e: e[2].record(stream)
        if consumer:
            ml.ml_magnification_map(h, ml.MAP_MU_F32, mu_out, stream)
            ml.ml_light_curves(h, tracks, TRACK_SAMPLES, SIGMA_PX, lc_out, stream)
            if args.workload == "fold":
                # the paper's light-curve statistics start from the 5 sigma peaks (§4.2)
                info_holder["peaks"] = ml.ml_find_peaks(h, ml.ALONG_X, 5.0, peak_mask, 0, stream)[0]
                # and bin them by distance beta_x from the caustic (Figs. 4-5)
                info_holder["peak_stats"] = ml.ml_peak_statistics(h, FOLD_DISTANCE_EDGES, ml.ALONG_X, 0.0,
                                                                  mask=peak_mask, stream=stream)
        if e: e[3].record(stream)
        # counters and the map's uint32 wrap-around check (a 64-bit map sum)
        stats, _ = ml.ml_field_stats(h, stream)
        if e: e[4].record(stream)
        ml.ml_field_destroy(h)
        info_holder["info"] = info
        info_holder["stats"] = stats
        if timers is not None:
            timers.append(e)
        return info, stats

    # the first step runs the autotuner (timed candidate builds and shots,
    # cached for the process): its create is reported apart, untimed in the step
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h0 = ml.ml_field_create(make_desc(True), stream)
    torch.cuda.synchronize()
    first_create_ms = (time.perf_counter() - t0) * 1e3
    ml.ml_field_destroy(h0)
    fp32_peak = measure_fp32_peak(ml, torch, stream, local, args.clocks_dir)
    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    timers = []
    with ClockSampler(local, args.clocks_dir) as clk:
        torch.cuda.synchronize()
        for _ in range(args.steps):
            flush.zero_()                 # L2 flush between timed steps (outside the events)
            step(timers)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    per = np.array([[a.elapsed_time(b) for a, b in zip(e[:-1], e[1:])] for e in timers])  # ms
    step_ms = float(per.sum(axis=1).mean())
    info, stats = info_holder["info"], info_holder["stats"]
    n_rays = info["n_rays_x"] * info["n_rays_y"]
    if args.shoot_rays:
        n_rays = int(min(args.shoot_rays, n_rays))
    t_local = step_ms
    if dist:
        t = torch.tensor([t_local], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_local = float(t.item())
    value = n_rays * (1 if sharded else world) / (t_local / 1e3)

    # roofline of the dominant kernel (the counting kernel)
    p = info["taylor_p"]
    shoot_ms = float(per[:, 1].mean())
    n_local = stats["rays_in"] + stats["rays_out"] + stats["rays_dropped"]   # this rank's rays
    expected_local = n_rays
    if sharded:
        a, b = shard.ray_ranges(info["n_rays_x"], info["n_rays_y"], info["n1y"], world)[rank]
        expected_local = b - a
    launches = max(1, stats["launches"])
    launch_s = shoot_ms / 1e3 / launches
    # the fixed algorithmic count per launch: 11 flop per near pair (Eq. 9's
    # near sum) + (8p + 10) per lattice ray (the degree-p series and the pixel)
    alg_flops = (11.0 * stats["near_pairs"] + (8.0 * p + 10.0) * n_local) / launches
    # the FP32 arithmetic actually executed: rays evaluated one by one (the
    # certified walk skips the rest), each its row polynomial as two real
    # Horner chains (4p), 6 for the pixel, 11 per near pair at the mean near
    # density (approximate for the evaluated rays)
    evals = stats.get("rays_evaluated", n_local)
    exec_flops = ((4.0 * p + 6.0) * evals + 11.0 * stats["near_pairs"] * evals / max(1, n_local)) / launches
    peak = fp32_peak["two_lane_tflops"]
    achieved = alg_flops / launch_s / 1e12
    traffic = traffic_per_launch(n_local / launches, args.workload, args.walk)
    hbm_peak, hbm_src = hbm_peak_gbs()
    out = {
        "metric": METRIC if args.workload == "paper" else
                  "rays/s of the Table-1 fold field (13,745 lenses) on 1 GB300; map L1 err vs FP64 oracle",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_local, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak", "vs_baseline": None,
        "dtype": "f32 (f64 node bases, c_0, sheet)",
        "data": "synthetic (seeded lognormal lens disc; no dataset)",
        "config": {"workload": w.name + f", {N_TRACKS} light curves x {TRACK_SAMPLES}",
                   "n_lenses": int(w.lenses.n), "n_rays": int(n_rays),
                   "map": f"{w.map_n[0]}x{w.map_n[1]} uint32",
                   "precision": "mixed: near sums, row series and c_1..c_p sums in FP32; node bases, "
                                "c_0 and the sheet in FP64",
                   "walk": args.walk, "certified_spans": bool(info["spans"]),
                   "span_far_lattice_units": info["span_far"] if info["span_far"] < 1e30 else "inf",
                   "build_flags": build_flags(),
                   "macro": "fold (Eq. 5)" if getattr(w, "macro", None) else "constant kappa, gamma (Eq. 1)",
                   "taylor_p": p, "far_bound_theta_e": info["far_bound"],
                   "l2_sub": [info["l2_sub_x"], info["l2_sub_y"]], "tuned_grid": bool(info["tuned"]),
                   "l1_theta_e": [info["n1x"] * info["l3x"], info["n1y"] * info["l3y"]],
                   "coefficient_build": {1: "direct", 2: "hierarchical"}.get(info["build"]),
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": (f"one map sharded over {world} GPUs (level-1 bands, integer "
                                   f"map sum onto rank 0)" if sharded else f"independent maps per GPU x{world}")},
        "breakdown_ms": {"create": float(per[:, 0].mean()), "shoot": shoot_ms,
                         ("mu_light_curves_and_peaks" if args.workload == "fold" else "mu_and_light_curves"):
                             float(per[:, 2].mean()),
                         "stats_and_wrap_check": float(per[:, 3].mean())},
        "first_create_with_autotuner_ms": first_create_ms,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "k_shoot_mixed",
                     "launch_ms": launch_s * 1e3,
                     "flops_per_launch": alg_flops,
                     "flop_count": "fixed count: 11 per near pair + (8p+10) per lattice ray",
                     "peak_note": "measured: ml_fp32_fma_peak two-lane FMA probe, best of 5 launches "
                                  f"at {fp32_peak.get('sm_mhz')} MHz (scalar FFMA "
                                  f"{fp32_peak['scalar_tflops']:.1f}, derived "
                                  f"{fp32_peak['derived_tflops_at_max_clock']:.1f} TFLOP/s)",
                     "executed": {"rays_evaluated_per_ray": evals / max(1, n_local),
                                  "flops_per_launch": exec_flops,
                                  "achieved": exec_flops / launch_s / 1e12,
                                  "frac": exec_flops / launch_s / 1e12 / peak},
                     "note": ("frac counts every lattice ray's fixed-convention work; the certified "
                              "walk evaluates only the rays_evaluated_per_ray fraction and proves the "
                              "others share an evaluated neighbour's pixel, so frac can exceed 1; "
                              "executed.frac is the pipe's share of the arithmetic it ran")
                             if args.walk == "certified" else None,
                     "hbm": ({"achieved_gbs": traffic / launch_s / 1e9, "peak_gbs": hbm_peak,
                              "frac": traffic / launch_s / 1e9 / hbm_peak, "peak_source": hbm_src}
                             if traffic else None)},
        "shoot_rays_override": bool(args.shoot_rays),
        **({"true_peaks_5sigma": info_holder.get("peaks"),
            "peak_statistics": fold_peak_summary(info_holder["peak_stats"], info)}
           if args.workload == "fold" and consumer else {}),
        "rays_check": {"in": stats["rays_in"], "out": stats["rays_out"],
                       "dropped": stats["rays_dropped"], "total": n_local,
                       "conserved": n_local == expected_local},
        "gpu_launches": int(args.steps * (BUILD_KERNELS + stats["launches"] + 1
                                          + (2 if consumer else 0)
                                          + (4 if args.workload == "fold" and consumer else 0))),
    }
    clk_sum = clk.summary()
    if clk_sum:
        out["clocks"] = clk_sum

    if not args.no_e2e:
        out["e2e"] = e2e(ml, w, torch, dev, stream, tracks, args, flush)

    oracle_run = None
    if rank == 0 and not args.no_parity:
        out["map_l1_vs_oracle"], oracle_run = parity_stripe(ml, w, stream, grid_kw)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the parity stripe's oracle run is a bounded sample of the same
        # workload: its timing is the CPU baseline when it ran
        out["cpu_baseline"] = (cpu_baseline_of(oracle_run, w) if oracle_run
                               else cpu_baseline(w))
    if sharded and not args.no_independent:
        # the same ranks, one map of their own each (no exchange): weak scaling
        out["independent_maps"] = independent_maps(ml, torch, w, grid_kw, stream, dev, rank, world, dist,
                                                   args, make_desc, inputs)
    if world == 1 and args.workload == "paper" and not args.no_sub:
        out["batched"] = run_batched(_sub_args(args), rank, world, local, compact=True)
        out["differentiable"] = run_differentiable(_sub_args(args), rank, world, local, compact=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return out


def _sub_args(args):
    """Arguments of the compact sub-records of the default line."""
    import copy
    a = copy.copy(args)
    a.steps, a.warmup = 2, 1
    a.no_e2e, a.no_cpu_baseline = True, True
    return a


def build_flags():
    """Extra nvcc flags the loaded library was built with ([] = the default)."""
    from paper_2308_14278_gb300 import build
    return build.built_flags()


def independent_maps(ml, torch, w0, grid_kw, stream, dev, rank, world, dist, args, make_desc, inputs):
    """Weak-scaling companion of a sharded run: each rank shoots a whole map
    of its own (seed = rank) with no data exchange; rays/s of the job."""
    w = inputs.paper_map(seed=rank, n_rays=args.rays, map_px=args.map_px, n_tracks=N_TRACKS)
    kw = dict(grid_kw)
    if args.grid:
        w.l1 = w0.l1
    times = []
    for k in range(1 + max(1, min(args.steps, 3))):
        f = ml.Field(w, precision=ml.PREC_MIXED, **kw)
        torch.cuda.synchronize()
        dist.barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f.shoot(stream=stream)
        e1.record(stream)
        e1.synchronize()
        if k > 0:
            times.append(e0.elapsed_time(e1))
        n = f.n_rays
        f.close()
    t = torch.tensor([float(np.mean(times))], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return {"value": n * world / (float(t.item()) / 1e3), "unit": UNIT, "scaling": "weak",
            "ms_per_shot": float(t.item()), "note": "shooting only (field build outside the events)"}


def e2e(ml, w, torch, dev, stream, tracks, args, flush):
    """The same step through the C ABI with host buffers: lens arrays from
    pinned host memory, map and light curves read back to pinned host memory."""
    pin = lambda a: torch.from_numpy(a).pin_memory()   # noqa: E731
    lx, ly, lm = pin(w.lenses.x), pin(w.lenses.y), pin(w.lenses.m)
    host = (lx.numpy(), ly.numpy(), lm.numpy())
    mu_h = torch.empty((w.map_n[1], w.map_n[0]), dtype=torch.float32).pin_memory().numpy()
    lc_h = torch.empty((N_TRACKS, TRACK_SAMPLES), dtype=torch.float32).pin_memory().numpy()

    grid_kw = grid_kwargs(args, w)

    def step():
        d = ml.make_desc(w, precision=ml.PREC_MIXED, lens_arrays=host, **grid_kw)
        h = ml.ml_field_create(d, stream)
        info = ml.ml_field_info(h)
        ml.ml_shoot_rays(h, 0, info["n_rays_x"] * info["n_rays_y"], stream)
        ml.ml_magnification_map(h, ml.MAP_MU_F32, mu_h, stream)
        ml.ml_light_curves(h, tracks, TRACK_SAMPLES, SIGMA_PX, lc_h, stream)
        ml.ml_field_destroy(h)
        return info["n_rays_x"] * info["n_rays_y"]

    step()
    times = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n = step()
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    return {"value": n / t, "unit": UNIT, "ms_per_step": t * 1e3,
            "h2d_bytes_per_step": int(3 * 8 * w.lenses.n + 32 * N_TRACKS),
            "d2h_bytes_per_step": int(4 * w.map_n[0] * w.map_n[1] + 4 * N_TRACKS * TRACK_SAMPLES)}


PARITY_STRIPE_RAYS = 10_000_000


def parity_stripe(ml, w, stream, grid_kw, n_rays: int = PARITY_STRIPE_RAYS):
    """Map relative L1 error vs the FP64 oracle on a stripe of n_rays
    consecutive lattice rays through the map's centre, shot alone, with the
    benchmark's grid.  Returns the result and the oracle run's
    (rays, seconds, threads, lattice rays)."""
    import oracle
    f = ml.Field(w, precision=ml.PREC_MIXED, **grid_kw)
    info = f.info
    g = oracle.geometry_of(w, p=info["taylor_p"], l2_sub=info["l2_sub_x"], l2_sub_y=info["l2_sub_y"],
                           l1=(info["n1x"] * info["l3x"], info["n1y"] * info["l3y"]))
    r0 = (g.n3y // 2) * g.n3x + 777
    r1 = min(g.n_rays, r0 + int(n_rays))
    f.shoot(r0, r1)
    got = f.counts().cpu().numpy().astype(np.int64)
    f.close()
    threads = oracle.default_threads()
    t0 = time.perf_counter()
    ref, _ = oracle.shoot_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, r0, r1, threads)
    dt = time.perf_counter() - t0
    l1 = float(np.abs(got - ref.astype(np.int64)).sum() / max(1, int(ref.sum())))
    return ({"value": l1, "stripe_rays": r1 - r0, "rays_in_map": int(ref.sum()),
             "pixels_differing": int(np.count_nonzero(got != ref)), "oracle_seconds": dt},
            (r1 - r0, dt, threads, g.n_rays))


def cpu_baseline_of(run, w):
    """The CPU baseline from the parity stripe's oracle run (FP64 direct sum
    as it stands, all host cores)."""
    n, dt, threads, lattice = run
    return {"value": n / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"the parity stripe: {n} consecutive rays of the {lattice:.3g}-ray lattice "
                      f"through all {w.lenses.n} lenses (FP64 direct sum, pthreads)", "seconds": dt}


def cpu_baseline(w, target_s: float = 12.0):
    """The FP64 oracle as it stands, on all host cores, on a bounded sample of
    the same workload: a contiguous stripe of rays through all 13,000 lenses."""
    import oracle
    g = oracle.geometry_of(w)
    r0 = (g.n3y // 3) * g.n3x
    threads = oracle.default_threads()
    n = 20000
    t0 = time.perf_counter()
    oracle.shoot_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, r0, r0 + n, threads)
    dt = time.perf_counter() - t0
    n2 = int(min(5e7, max(n, n * target_s / max(dt, 1e-3))))
    t0 = time.perf_counter()
    oracle.shoot_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, r0, r0 + n2, threads)
    dt = time.perf_counter() - t0
    return {"value": n2 / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n2} consecutive rays of the {g.n_rays:.3g}-ray lattice through all "
                      f"{w.lenses.n} lenses (FP64 direct sum, pthreads)", "seconds": dt}


# ---------------------------------------------------------------------------
# batched maps: one graph-captured persistent launch over 80 maps
# ---------------------------------------------------------------------------

def _events(torch, n):
    return [torch.cuda.Event(enable_timing=True) for _ in range(n)]


def run_batched(args, rank, world, local, compact=False):
    """80 heterogeneous maps (2,000-20,000 lenses, 1e9-1e10 rays, 4096^2) and
    their 800 light curves as one CUDA-graph replay of the batched launch,
    next to the same maps shot one at a time, both with the batch's own
    (autotuned) grids and orders and with Eq. 10's grids.  compact: the
    sub-record of the default line (no e2e, no CPU baseline, no NCCL)."""
    import torch
    torch.cuda.set_device(local)
    import paper_2308_14278_gb300 as ml
    from paper_2308_14278_gb300 import inputs, shard
    ml.load()
    dist = None
    if world > 1 and not compact:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    # N > 1: the ranks split one set of 80 maps (whole maps, balanced by
    # rays, nothing exchanged); --independent: each rank runs its own 80 maps
    sharded = bool(dist is not None and not args.independent)
    seed = 0 if sharded else rank
    n_all, tpm, map_px = 80, 10, 4096
    ws = inputs.batched_maps(n_maps=n_all, seed=seed, map_px=map_px, ray_range=(1e9, 1e10),
                             tracks_per_map=tpm)
    tracks = np.stack([inputs.tracks(tpm, map_px, map_px, 4 * SIGMA_PX + 1, seed=500 + 100 * seed + i)
                       for i in range(n_all)])
    if sharded:
        mine = shard.maps_for_rank([w.n_av * w.map_n[0] * w.map_n[1] for w in ws], rank, world)
        ws, tracks = [ws[i] for i in mine], tracks[mine]
    n_maps = len(ws)
    stream = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    walk = ml.WALK_PER_RAY if args.walk == "per_ray" else ml.WALK_CERTIFIED
    t0 = time.perf_counter()
    descs = [ml.make_desc(w, precision=ml.PREC_MIXED, tune=True, walk=walk) for w in ws]
    b = ml.Batch(descs, tracks=tracks, n_samples=TRACK_SAMPLES, sigma_px=SIGMA_PX)
    torch.cuda.synchronize()
    create_s = time.perf_counter() - t0
    infos = [b.info(i) for i in range(n_maps)]
    rays = sum(i["n_rays_x"] * i["n_rays_y"] for i in infos)
    orders = sorted({i["taylor_p"] for i in infos})
    for _ in range(args.warmup):
        b.run(use_graph=True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    times = []
    with ClockSampler(local, args.clocks_dir, tag="_batched") as clk:
        for _ in range(args.steps):
            flush.zero_()
            e = _events(torch, 2)
            e[0].record(stream)
            b.run(use_graph=True)
            e[1].record(stream)
            times.append(e)
        torch.cuda.synchronize()
    step_ms = float(np.mean([a.elapsed_time(c) for a, c in times]))
    stats = [b.stats(i) for i in range(n_maps)]
    t_local = step_ms
    rays_job = rays * world
    if dist:
        t = torch.tensor([t_local], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_local = float(t.item())
        if sharded:
            r = torch.tensor([rays], device="cuda", dtype=torch.int64)
            dist.all_reduce(r)
            rays_job = int(r.item())
    value = rays_job / (t_local / 1e3)

    # the same maps one at a time: (a) each with the batch's grid and order,
    # (b) each with Eq. 10's level-1 cells and the paper's level-2 grid
    mu1 = torch.empty((map_px, map_px), dtype=torch.float32, device="cuda")
    lc1 = torch.empty((tpm, TRACK_SAMPLES), dtype=torch.float32, device="cuda")

    def one_at_a_time(fields):
        for f, tr in zip(fields, tracks):
            f.clear(stream)
            f.shoot(stream=stream)
            ml.ml_magnification_map(f.h, ml.MAP_MU_F32, mu1, stream)
            ml.ml_light_curves(f.h, tr, TRACK_SAMPLES, SIGMA_PX, lc1, stream)

    def time_fields(fields):
        one_at_a_time(fields)
        single = []
        for _ in range(max(1, min(args.steps, 2))):
            flush.zero_()
            e = _events(torch, 2)
            e[0].record(stream)
            one_at_a_time(fields)
            e[1].record(stream)
            torch.cuda.synchronize()
            single.append(e[0].elapsed_time(e[1]))
        return float(np.mean(single))

    same = [ml.Field(w, precision=ml.PREC_MIXED, walk=walk, taylor_p=i["taylor_p"],
                     l1=(i["n1x"] * i["l3x"], i["n1y"] * i["l3y"]), l2_sub=(i["l2_sub_x"], i["l2_sub_y"]),
                     span_far=i["span_far"])
            for w, i in zip(ws, infos)]
    same_ms = time_fields(same)
    # the batch's map 0 against the same map shot alone with the same grid
    b.run(use_graph=True)
    same[0].clear(stream)
    same[0].shoot(stream=stream)
    batch_equals_single = bool(torch.equal(b.counts(0), same[0].counts()))
    for f in same:
        f.close()
    paper = [ml.Field(w, precision=ml.PREC_MIXED, walk=walk) for w in ws]
    paper_ms = time_fields(paper)
    paper_p = sorted({f.info["taylor_p"] for f in paper})
    for f in paper:
        f.close()

    # map error against the oracle: a stripe of map 0 shot alone on its batch grid
    map_err = None
    if rank == 0 and not args.no_parity:
        w0, i0 = ws[0], infos[0]
        w0.l1 = (i0["n1x"] * i0["l3x"], i0["n1y"] * i0["l3y"])
        map_err, _ = parity_stripe(ml, w0, stream, dict(l2_sub=(i0["l2_sub_x"], i0["l2_sub_y"]),
                                                        taylor_p=i0["taylor_p"], walk=walk),
                                   n_rays=200_000)

    fixed = sum(11.0 * st["near_pairs"] + (8.0 * i["taylor_p"] + 10.0) * i["n_rays_x"] * i["n_rays_y"]
                for st, i in zip(stats, infos))
    evals = sum(st["rays_evaluated"] for st in stats)
    fp32_peak = measure_fp32_peak(ml, torch, stream, local, args.clocks_dir, launches=3)
    peak = fp32_peak["two_lane_tflops"]
    achieved = fixed / (step_ms / 1e3) / 1e12
    out = {
        "metric": "rays/s of 80 batched maps on 1 GB300 (one CUDA graph: a persistent launch per Taylor order)",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_local, "higher_is_better": True, "scaling": "strong" if sharded else "weak",
        "vs_baseline": None,
        "dtype": "f32 (f64 node bases, c_0, sheet)", "data": "synthetic (seeded lognormal lens discs; no dataset)",
        "config": {"workload": f"batched: {n_all} maps, 2,000-20,000 lenses, kappa_* in "
                               f"{{0.002, 0.005, 0.01}}, kappa+gamma 0.95-0.99, 1e9-1e10 rays each, "
                               f"{map_px}^2 uint32, {n_all * tpm} light curves x {TRACK_SAMPLES}",
                   "total_rays": int(rays_job if sharded else rays), "taylor_p": orders, "tuned_grids": True,
                   "walk": args.walk, "launches_per_step": len(orders),
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": (f"one set of {n_all} maps split over {world} GPUs (whole maps, "
                                   f"balanced by rays)" if sharded else f"independent batches per GPU x{world}")},
        "create_s": create_s,
        "one_map_at_a_time_same_grids": {"ms_per_step": same_ms, "value": rays / (same_ms / 1e3),
                                         "speedup_of_batched": same_ms / step_ms},
        "one_map_at_a_time_eq10_grids": {"ms_per_step": paper_ms, "value": rays / (paper_ms / 1e3),
                                         "taylor_p": paper_p, "speedup_of_batched": paper_ms / step_ms},
        "batch_map_equals_single_map": batch_equals_single,
        "map_l1_vs_oracle": map_err,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "k_shoot_batch",
                     "rays_evaluated_per_ray": evals / max(1, rays),
                     "note": "whole graph step time (clear, shoot, mu, curves) as the kernel time; "
                             "the fixed flop count per lattice ray (11 per near pair + (8p+10))",
                     "peak_note": "measured: ml_fp32_fma_peak two-lane FMA probe"},
        "rays_check": {"conserved": all(st["rays_in"] + st["rays_out"] + st["rays_dropped"] ==
                                        i["n_rays_x"] * i["n_rays_y"] for st, i in zip(stats, infos))},
        "gpu_launches": int(args.steps * (len(orders) + 2 * n_maps)),
    }
    clk_sum = clk.summary()
    if clk_sum:
        out["clocks"] = clk_sum
    if not args.no_e2e:
        # through the public API from host buffers: create from host lens arrays,
        # run, read the 800 light curves back to pinned host memory
        curves_h = torch.empty((n_maps, tpm, TRACK_SAMPLES), dtype=torch.float32).pin_memory()
        b.close()
        te = []
        for _ in range(max(1, min(args.steps, 2))):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            bb = ml.Batch([ml.make_desc(w, precision=ml.PREC_MIXED, tune=True, walk=walk) for w in ws],
                          tracks=tracks, n_samples=TRACK_SAMPLES, sigma_px=SIGMA_PX)
            bb.run(use_graph=True)
            ml._check(ml.load().ml_batch_curves(bb.h, curves_h.numpy().ctypes.data, 0, None))
            torch.cuda.synchronize()
            te.append(time.perf_counter() - t0)
            bb.close()
        t = float(np.mean(te))
        if dist:
            tt = torch.tensor([t], device="cuda", dtype=torch.float64)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            t = float(tt.item())
        out["e2e"] = {"value": rays_job / t, "unit": UNIT, "ms_per_step": t * 1e3,
                      "h2d_bytes_per_step": int(sum(24 * w.lenses.n for w in ws) + tracks.nbytes),
                      "d2h_bytes_per_step": int(4 * n_maps * tpm * TRACK_SAMPLES),
                      "note": "includes batch creation (tuned grids cached per process)"}
    else:
        b.close()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(ws[0], target_s=10.0)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if compact:
        keep = ("value", "unit", "ms_per_step", "create_s", "one_map_at_a_time_same_grids",
                "one_map_at_a_time_eq10_grids", "batch_map_equals_single_map", "map_l1_vs_oracle",
                "roofline", "rays_check")
        out = {k: out[k] for k in keep} | {"config": {"workload": out["config"]["workload"],
                                                       "taylor_p": orders, "launches_per_step": len(orders)}}
    return out


# ---------------------------------------------------------------------------
# differentiable map: CIC forward + hand-written adjoint
# ---------------------------------------------------------------------------

def run_differentiable(args, rank, world, local, compact=False):
    """One optimisation step of a lens field against a target map: create the
    field from device lens arrays, the CIC map (ml_cic_forward), dL/dM of
    L = |M - T|^2, and the adjoint (ml_cic_backward) to d/d(x_k, y_k, m_k,
    kappa, gamma, kappa_*).  1,000 lenses, 4e8 rays, 1024^2 float32."""
    import torch
    torch.cuda.set_device(local)
    import paper_2308_14278_gb300 as ml
    from paper_2308_14278_gb300 import inputs
    ml.load()
    dist = None
    if world > 1 and not compact:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = inputs.differentiable_field(seed=rank)
    wt = inputs.differentiable_field(seed=rank + 1000)        # target from a perturbed seed
    stream = torch.cuda.current_stream()
    dev = torch.device("cuda", local)
    ny, nx = w.map_n[1], w.map_n[0]
    T = torch.empty((ny, nx), dtype=torch.float32, device=dev)
    ft = ml.Field(wt, precision=ml.PREC_MIXED, deposit=ml.DEPOSIT_CIC)
    ml.ml_cic_forward(ft.h, T)
    ft.close()
    lens_dev = [torch.from_numpy(a).to(dev) for a in (w.lenses.x, w.lenses.y, w.lenses.m)]
    mu = torch.empty((ny, nx), dtype=torch.float32, device=dev)
    G = torch.empty_like(mu)
    gl = torch.empty((w.lenses.n, 3), dtype=torch.float64, device=dev)
    gp = torch.empty(3, dtype=torch.float64, device=dev)
    loss = torch.empty((), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def desc(lens=None):
        d = ml.make_desc(w, precision=ml.PREC_MIXED, deposit=ml.DEPOSIT_CIC)
        d.lens_x, d.lens_y, d.lens_m = (t.data_ptr() for t in (lens or lens_dev))
        d.lens_mem_is_device = 1
        return d

    hold = {}

    def step(e=None):
        if e: e[0].record(stream)
        h = ml.ml_field_create(desc(), stream)
        if e: e[1].record(stream)
        ml.ml_cic_forward(h, mu, stream)
        if e: e[2].record(stream)
        torch.sub(mu, T, out=G)                       # dL/dM = 2 (M - T), the caller's loss
        torch.sum(G.double() ** 2, dim=(0, 1), out=loss)
        G.mul_(2.0)
        if e: e[3].record(stream)
        ml.ml_cic_backward(h, G, gl, gp, stream)
        if e: e[4].record(stream)
        hold["info"] = ml.ml_field_info(h)
        hold["stats"] = ml.ml_field_stats(h, stream)[0]
        ml.ml_field_destroy(h)

    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    timers = []
    with ClockSampler(local, args.clocks_dir, tag="_differentiable") as clk:
        for _ in range(args.steps):
            flush.zero_()
            e = _events(torch, 5)
            step(e)
            timers.append(e)
        torch.cuda.synchronize()
    per = np.array([[a.elapsed_time(c) for a, c in zip(e[:-1], e[1:])] for e in timers])
    # finite-difference spot check of one gradient component: the lens at least
    # 0.3 theta_E outside the ray rectangle with the largest |dL/dx|, central
    # differences of the loss through the library's forward at h = 3e-4
    gl_h = gl.cpu().numpy()

    def loss_of(lens):
        h = ml.ml_field_create(desc(lens), stream)
        ml.ml_cic_forward(h, mu, stream)
        v = float(((mu.double() - T.double()) ** 2).sum().item())
        ml.ml_field_destroy(h)
        return v

    rb = hold["info"]
    x0, y0, x1, y1 = rb["ray_x0"], rb["ray_y0"], rb["ray_x1"], rb["ray_y1"]
    dist_out = np.hypot(np.maximum(np.maximum(x0 - w.lenses.x, w.lenses.x - x1), 0),
                        np.maximum(np.maximum(y0 - w.lenses.y, w.lenses.y - y1), 0))
    k = int(np.argmax(np.where(dist_out > 0.3, np.abs(gl_h[:, 0]), -1.0)))
    hfd = 3e-4
    base = [loss_of(None) for _ in range(3)]
    xp, xm = lens_dev[0].clone(), lens_dev[0].clone()
    xp[k] += hfd
    xm[k] -= hfd
    fd = (loss_of([xp, lens_dev[1], lens_dev[2]]) - loss_of([xm, lens_dev[1], lens_dev[2]])) / (2 * hfd)
    fd_check = {"lens": k, "component": "x", "h": hfd, "finite_difference": fd, "adjoint": float(gl_h[k, 0]),
                "rel_diff": abs(fd - gl_h[k, 0]) / max(abs(gl_h[k, 0]), 1e-300),
                "loss_spread_over_2h": (max(base) - min(base)) / (2 * hfd)}
    step_ms = float(per.sum(axis=1).mean())
    info, stats = hold["info"], hold["stats"]
    n_rays = info["n_rays_x"] * info["n_rays_y"]
    t_local = step_ms
    if dist:
        t = torch.tensor([t_local], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_local = float(t.item())
    value = n_rays * world / (t_local / 1e3)
    p = info["taylor_p"]
    bw_ms = float(per[:, 3].mean())
    live = stats["rays_in"] / max(1, n_rays)
    pairs = stats["near_pairs"]
    # adjoint work: the forward recomputed (11 per near pair + 4p + 6 per ray),
    # then per live ray the CIC gradient and node moments (5p + 25) and 15 per
    # near pair in the near pass
    flops = 11.0 * pairs + (4.0 * p + 6.0) * n_rays + live * (15.0 * pairs + (5.0 * p + 25.0) * n_rays)
    achieved = flops / (bw_ms / 1e3) / 1e12
    fp32_peak = measure_fp32_peak(ml, torch, stream, local, args.clocks_dir, launches=3)
    peak = fp32_peak["two_lane_tflops"]
    peak_note = "measured: ml_fp32_fma_peak two-lane FMA probe"
    out = {
        "metric": "rays/s of a CIC forward + adjoint step (1,000 lenses, 4e8 rays) on 1 GB300",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_local, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32 (f64 node bases, c_0, sheet; f64 gradient sums)",
        "data": "synthetic (seeded lognormal lens disc; target map from seed + 1000)",
        "config": {"workload": w.name + ", loss |M - T|^2, gradient w.r.t. all lenses, kappa, gamma, "
                               "kappa_*", "n_lenses": int(w.lenses.n), "n_rays": int(n_rays),
                   "taylor_p": p, "far_bound_theta_e": info["far_bound"],
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"independent fields per GPU x{world}"},
        "breakdown_ms": {"create": float(per[:, 0].mean()), "forward": float(per[:, 1].mean()),
                         "loss": float(per[:, 2].mean()), "backward": bw_ms},
        "loss": float(loss.item()),
        "gradient_fd_check": fd_check,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "k_adj_rays + k_adj_far",
                     "peak_note": peak_note},
        "gpu_launches": int(args.steps * (BUILD_KERNELS + 2 + 3)),
    }
    clk_sum = clk.summary()
    if clk_sum:
        out["clocks"] = clk_sum
    if not args.no_e2e:
        host = (w.lenses.x, w.lenses.y, w.lenses.m)
        gl_h = torch.empty((w.lenses.n, 3), dtype=torch.float64).pin_memory()
        gp_h = torch.empty(3, dtype=torch.float64).pin_memory()
        te = []
        for _ in range(max(1, min(args.steps, 3))):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = ml.ml_field_create(ml.make_desc(w, precision=ml.PREC_MIXED, deposit=ml.DEPOSIT_CIC,
                                                lens_arrays=host), stream)
            ml.ml_cic_forward(h, mu, stream)
            torch.sub(mu, T, out=G)
            torch.sum(G.double() ** 2, dim=(0, 1), out=loss)
            G.mul_(2.0)
            ml.ml_cic_backward(h, G, gl, gp, stream)
            gl_h.copy_(gl, non_blocking=True)
            gp_h.copy_(gp, non_blocking=True)
            lv = float(loss.item())
            ml.ml_field_destroy(h)
            torch.cuda.synchronize()
            te.append(time.perf_counter() - t0)
        t = float(np.mean(te))
        out["e2e"] = {"value": n_rays / t, "unit": UNIT, "ms_per_step": t * 1e3,
                      "h2d_bytes_per_step": int(24 * w.lenses.n),
                      "d2h_bytes_per_step": int(gl_h.numel() * 8 + 24 + 8), "loss": lv}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline_grad(w, ml)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if compact:
        keep = ("value", "unit", "ms_per_step", "breakdown_ms", "loss", "gradient_fd_check", "roofline")
        out = {k: out[k] for k in keep} | {"config": {"workload": out["config"]["workload"]}}
    return out


def cpu_baseline_grad(w, ml, target_s: float = 10.0):
    """The oracle's FP64 CIC gradient (every ray against every lens) on all
    host cores, on a contiguous block of rays of the same lattice."""
    import oracle
    g = oracle.geometry_of(w)
    threads = oracle.default_threads()
    T = np.zeros((g.mny, g.mnx))
    r0 = (g.n3y // 2) * g.n3x
    n = 200000
    t0 = time.perf_counter()
    oracle.cic_grad(g, w.lenses.x, w.lenses.y, w.lenses.m, T, r0, r0 + n, threads)
    dt = time.perf_counter() - t0
    n2 = int(min(5e7, max(n, n * target_s / max(dt, 1e-3))))
    t0 = time.perf_counter()
    oracle.cic_grad(g, w.lenses.x, w.lenses.y, w.lenses.m, T, r0, r0 + n2, threads)
    dt = time.perf_counter() - t0
    return {"value": n2 / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"{n2} consecutive rays of the {g.n_rays:.3g}-ray lattice: CIC map and "
                      f"FP64 gradient against all {w.lenses.n} lenses", "seconds": dt}


# ---------------------------------------------------------------------------
# reference arm: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def run_reference(args, rank, world):
    if rank != 0:
        return None
    import oracle
    from paper_2308_14278_gb300 import inputs
    oracle.build()
    w = inputs.paper_map(seed=0, n_rays=args.rays, map_px=args.map_px, n_tracks=N_TRACKS)
    g = oracle.geometry_of(w)
    threads = oracle.default_threads()
    # size one step at ~8 s of CPU work so that warm-up + steps stay within minutes
    n = 20000
    r0 = (g.n3y // 3) * g.n3x
    t0 = time.perf_counter()
    oracle.shoot_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, r0, r0 + n, threads)
    per = max(time.perf_counter() - t0, 1e-3) / n
    n_step = int(max(n, min(2e7, 8.0 / per)))
    for _ in range(args.warmup):
        oracle.shoot_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, r0, r0 + min(n_step, 20000),
                            threads)
    times = []
    for k in range(args.steps):
        a = r0 + k * n_step
        t0 = time.perf_counter()
        oracle.shoot_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, a, a + n_step, threads)
        times.append(time.perf_counter() - t0)
    t = float(np.mean(times))
    value = n_step / t
    sample = (f"{n_step} consecutive rays per step of the {g.n_rays:.3g}-ray lattice through "
              f"all {w.lenses.n} lenses (FP64 direct sum)")
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded lognormal lens disc; no dataset)",
            "config": {"workload": w.name, "n_lenses": int(w.lenses.n), "n_rays": int(g.n_rays),
                       "map": f"{w.map_n[0]}x{w.map_n[1]}", "precision": "fp64 direct sum"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.fp32_peak_only:
        import torch
        torch.cuda.set_device(local)
        import paper_2308_14278_gb300 as ml
        ml.load()
        res = {}
        for bps in (1, 2, 4, 8):
            sink = torch.zeros(8 * 1024, dtype=torch.float32, device=f"cuda:{local}")
            for two in (False, True):
                best = 0.0
                for _ in range(3):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    st = torch.cuda.current_stream()
                    e0.record(st)
                    flop = ml.ml_fp32_fma_peak(two, bps, PEAK_ITERS // 2, sink, st)
                    e1.record(st)
                    e1.synchronize()
                    best = max(best, flop / (e0.elapsed_time(e1) / 1e3) / 1e12)
                res[f"{bps}_blocks_per_sm_{'two_lane' if two else 'scalar'}_tflops"] = best
        res["bench_measurement"] = measure_fp32_peak(ml, torch, torch.cuda.current_stream(), local,
                                                     args.clocks_dir)
        print(json.dumps(res), flush=True)
        return
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    elif args.workload == "batched":
        out = run_batched(args, rank, world, local)
    elif args.workload == "differentiable":
        out = run_differentiable(args, rank, world, local)
    else:
        out = run_ours(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
