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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "rays/s at 13k lenses on 1 GB300; % FP32 peak; map L1 err vs FP64 oracle"
UNIT = "rays/s"
N_TRACKS, TRACK_SAMPLES, SIGMA_PX = 10, 4096, 0.5
# FP32 FMA units of GB300 (152 SMs x 128 lanes) at the maximum SM clock
SMS, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
# DRAM bytes per ray of the shooting kernel, from the ncu capture summarised in
# profiles/k_shoot_mixed_paper-map-2e10-ray-slice.md (dram__bytes_read.sum +
# dram__bytes_write.sum = 450.4 MB for 2.0e10 rays), valid for the kernel
# sources with these sha1 prefixes only.
TRAFFIC_BYTES_PER_RAY = 450.413056e6 / 2.0e10
TRAFFIC_SOURCES = {"ml_shoot.cu": "26dd64ff", "ml_internal.cuh": "9b6a32ff"}


def traffic_per_launch(rays_per_launch: float):
    """Measured DRAM bytes per launch, or None once the kernel has changed."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2308_14278_gb300", "csrc")
    for name, prefix in TRAFFIC_SOURCES.items():
        with open(os.path.join(csrc, name), "rb") as fh:
            if not hashlib.sha1(fh.read()).hexdigest().startswith(prefix):
                return None
    return TRAFFIC_BYTES_PER_RAY * rays_per_launch


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--rays", type=float, default=1e11)
    ap.add_argument("--map-px", type=int, default=8192)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-parity", action="store_true")
    ap.add_argument("--shoot-rays", type=float, default=0,
                    help="profiling: shoot only this many rays (a centred slice of the lattice) "
                         "per step; the default shoots them all")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}",
                                          f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.send_signal(signal.SIGTERM)
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        load = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": float(np.median(load)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# our implementation
# ---------------------------------------------------------------------------

def run_ours(args, rank, world, local):
    import torch
    torch.cuda.set_device(local)
    import paper_2308_14278_gb300 as ml
    from paper_2308_14278_gb300 import inputs
    ml.load()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # weak scaling: every rank makes its own map (own seed) of the same size
    w = inputs.paper_map(seed=rank, n_rays=args.rays, map_px=args.map_px, n_tracks=N_TRACKS)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    lens_dev = [torch.from_numpy(a).to(dev) for a in (w.lenses.x, w.lenses.y, w.lenses.m)]
    tracks = inputs.tracks(N_TRACKS, w.map_n[0], w.map_n[1], 4 * SIGMA_PX + 1, seed=100 + rank)
    mu_out = torch.empty((w.map_n[1], w.map_n[0]), dtype=torch.float32, device=dev)
    lc_out = torch.empty((N_TRACKS, TRACK_SAMPLES), dtype=torch.float32, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)   # > L2 (129 MB)

    def make_desc(device_lenses: bool, host_lenses=None):
        d = ml.make_desc(w, precision=ml.PREC_MIXED, lens_arrays=host_lenses)
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
        ml.ml_shoot_rays(h, r0, r0 + n_shoot, stream)
        if e: e[2].record(stream)
        ml.ml_magnification_map(h, ml.MAP_MU_F32, mu_out, stream)
        if e: e[3].record(stream)
        ml.ml_light_curves(h, tracks, TRACK_SAMPLES, SIGMA_PX, lc_out, stream)
        if e: e[4].record(stream)
        stats, _ = ml.ml_field_stats(h, stream)
        ml.ml_field_destroy(h)
        info_holder["info"] = info
        info_holder["stats"] = stats
        if timers is not None:
            timers.append(e)
        return info, stats

    for _ in range(args.warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    timers = []
    with ClockSampler(local) as clk:
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
    value = n_rays * world / (t_local / 1e3)

    # roofline of the dominant kernel (the shooting kernel): algorithmic FP32
    # work per ray of this algorithm = 11 per near pair + 4p (two real Horner
    # polynomials of degree p) + 6 (near fold, binning)
    p = info["taylor_p"]
    shoot_ms = float(per[:, 1].mean())
    flops = 11.0 * stats["near_pairs"] + (4.0 * p + 6.0) * n_rays
    achieved = flops / (shoot_ms / 1e3) / 1e12
    peak = SMS * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12
    survey_flops = 11.0 * stats["near_pairs"] + (8.0 * p + 10.0) * n_rays

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_local, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 near sum + f64 nodes",
        "data": "synthetic (seeded lognormal lens disc; no dataset)",
        "config": {"workload": w.name + f", {N_TRACKS} light curves x {TRACK_SAMPLES}",
                   "n_lenses": int(w.lenses.n), "n_rays": int(n_rays),
                   "map": f"{w.map_n[0]}x{w.map_n[1]} uint32", "precision": "mixed",
                   "taylor_p": p, "far_bound_theta_e": info["far_bound"],
                   "coefficient_build": {1: "direct", 2: "hierarchical"}.get(info["build"]),
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": f"independent maps per GPU x{world}"},
        "breakdown_ms": {"create": float(per[:, 0].mean()), "shoot": shoot_ms,
                         "mu": float(per[:, 2].mean()), "light_curves": float(per[:, 3].mean())},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": traffic_per_launch(n_rays / max(1, stats["launches"])),
                     "kernel": "k_shoot_mixed", "flops_per_launch_survey_convention":
                         survey_flops / max(1, stats["launches"]),
                     "peak_note": "152 SMs x 128 FP32 lanes x 2 x 2070 MHz (derived)"},
        "shoot_rays_override": bool(args.shoot_rays),
        "rays_check": {"in": stats["rays_in"], "out": stats["rays_out"],
                       "dropped": stats["rays_dropped"], "total": n_rays,
                       "conserved": stats["rays_in"] + stats["rays_out"] + stats["rays_dropped"] == n_rays},
        "gpu_launches": int(args.steps * (6 + stats["launches"] + 2)),
    }
    clk_sum = clk.summary()
    if clk_sum:
        out["clocks"] = clk_sum

    if not args.no_e2e:
        out["e2e"] = e2e(ml, w, torch, dev, stream, tracks, args, flush)

    if rank == 0 and not args.no_parity:
        out["map_l1_vs_oracle"] = parity_stripe(ml, w, stream)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(w)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return out


def e2e(ml, w, torch, dev, stream, tracks, args, flush):
    """The same step through the C ABI with host buffers: lens arrays from
    pinned host memory, map and light curves read back to pinned host memory."""
    pin = lambda a: torch.from_numpy(a).pin_memory()   # noqa: E731
    lx, ly, lm = pin(w.lenses.x), pin(w.lenses.y), pin(w.lenses.m)
    host = (lx.numpy(), ly.numpy(), lm.numpy())
    mu_h = torch.empty((w.map_n[1], w.map_n[0]), dtype=torch.float32).pin_memory().numpy()
    lc_h = torch.empty((N_TRACKS, TRACK_SAMPLES), dtype=torch.float32).pin_memory().numpy()

    def step():
        d = ml.make_desc(w, precision=ml.PREC_MIXED, lens_arrays=host)
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


def parity_stripe(ml, w, stream):
    """Map relative L1 error vs the FP64 oracle on a stripe of 1e6 rays shot alone."""
    import oracle
    f = ml.Field(w, precision=ml.PREC_MIXED)
    g = oracle.geometry_of(w, p=f.info["taylor_p"])
    r0 = (g.n3y // 2) * g.n3x + 777
    r1 = r0 + 1_000_000
    f.shoot(r0, r1)
    got = f.counts().cpu().numpy().astype(np.int64)
    f.close()
    t0 = time.perf_counter()
    ref, _ = oracle.shoot_direct(g, w.lenses.x, w.lenses.y, w.lenses.m, r0, r1)
    l1 = float(np.abs(got - ref.astype(np.int64)).sum() / max(1, int(ref.sum())))
    return {"value": l1, "stripe_rays": r1 - r0, "rays_in_map": int(ref.sum()),
            "oracle_seconds": time.perf_counter() - t0}


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
    if args.impl == "reference":
        out = run_reference(args, rank, world)
    else:
        out = run_ours(args, rank, world, local)
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
