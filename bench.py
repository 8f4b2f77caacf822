#!/usr/bin/env python3
"""Benchmark of the embedded-gasket hot path on GB300.

Headline (one JSON line on stdout): the lambda-mapped map-and-write pass on a
level-16 gasket embedded in a 65536 x 65536 uint8 grid (4.3 GB), value = hash
of (x, y) with seed 1.  A step is one pass over the whole grid; the metric is
gasket cells written per second (3^16 cells per pass).  The grid (4.3 GB) and
the sectors one pass touches (181 MB) are both larger than the 129 MB L2, so
no L2 flush is needed between passes.

Beside the headline the line carries: the roofline of the write kernel
(touched 128-byte lines per launch / CUDA-event launch time, against the
measured HBM copy bandwidth), the bounding-box map on the same workload, the
float32 grid, the level-15 CA and diffusion steps (single and fused), the
compact layout's write pass and steps, the level sweep, the batched CA and
the continuous-batching server, the end-to-end rate through host buffers,
SM clocks sampled during the run, and the CPU oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (the only reference this method has)
on the same workload.  A step gives every host core one band of 1024 rows of
the level-16 grid, run side by side in spawned processes (16 bands per step
on a 16-core host); successive steps move on through the grid's 64 bands.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = ("gasket GCells/s and % of HBM peak at n=2^16, λ vs bounding-box; "
          "served p50/p99 latency")
UNIT = "GCells/s"
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 8000.0


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--rho", type=int, default=None)
    p.add_argument("--map", default=None)
    p.add_argument("--order", default=None, choices=("rowmajor", "interleaved"))
    p.add_argument("--store", default=None, choices=("auto", "scatter", "staged", "tma", "fill",
                                                     "sector", "merge", "masked"))
    p.add_argument("--value", default=None, choices=("hash", "linear31", "const"),
                   help="with --quick: the written value (a constant times the store path "
                        "alone)")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the comparison workloads (bbox, f32, stencils)")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--quick", action="store_true",
                   help="headline launches only (no clock soak, extras, e2e or CPU "
                        "baseline): the form used under ncu")
    p.add_argument("--write-sweep", action="store_true",
                   help="the map-and-write sweep instead of the headline: levels 8..16, "
                        "uint8 and float32, rho 8..64, lambda vs bounding box; prints one "
                        "JSON line")
    p.add_argument("--paper-sweep", action="store_true",
                   help="the paper's experiment instead of the headline: write a constant "
                        "into the gasket of a zero uint8 matrix for r = 0..16, rho = 1..32, "
                        "lambda (bounding sub-boxes, per-cell stores) vs bounding box, timed "
                        "as 100 sub-averages of 10 consecutive calls; prints one JSON line")
    p.add_argument("--workload", choices=("write", "ca", "diffusion", "ca_fused",
                                          "diffusion_fused", "ca_compact",
                                          "diffusion_compact", "ca_compact_fused",
                                          "batch_ca_fused", "serve_fused"),
                   default="write",
                   help="with --quick: time the level-15 CA or diffusion step (or its "
                        "fused form, k steps per launch), or the batch of 64 gaskets' "
                        "16-step fused launch (batch_ca_fused), or a saturated serving "
                        "trace (serve_fused), instead of the write pass "
                        "(the form used to profile those kernels)")
    p.add_argument("--level", type=int, default=None,
                   help="with --quick: the gasket level (stencils: default 15; write: 16)")
    p.add_argument("--dtype", default="u8", choices=("u8", "f32"),
                   help="with --quick and the write workload: the grid's element type")
    p.add_argument("--staging", default=None, choices=("chunks", "tma"),
                   help="with --quick and the ca / diffusion workloads: how tiles are staged")
    p.add_argument("--l2-fetch", type=int, default=None,
                   help="with --quick: run with this L2 fetch granularity (bytes) as the "
                        "context's limit")
    return p.parse_args()


# --------------------------------------------------------------------------
# process group (N > 1: independent replicas, one per GPU)
# --------------------------------------------------------------------------
class Group:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.dist = None
        self.backend = None
        if self.world > 1:
            import torch.distributed as dist
            # SG_BENCH_BACKEND=gloo keeps every rank on the CPU (used by tests)
            self.backend = os.environ.get("SG_BENCH_BACKEND") or (
                "nccl" if _cuda_ok() else "gloo")
            if self.backend == "nccl":
                import torch
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend=self.backend)
            self.dist = dist

    def barrier(self):
        if self.dist is not None:
            self.dist.barrier()

    def max(self, value: float) -> float:
        if self.dist is None:
            return value
        import torch
        dev = f"cuda:{self.local}" if self.backend == "nccl" else "cpu"
        t = torch.tensor([value], dtype=torch.float64, device=dev)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.dist is not None:
            self.dist.destroy_process_group()


def _cuda_ok() -> bool:
    try:
        import torch
        return torch.cuda.is_available()
    except Exception:
        return False


# --------------------------------------------------------------------------
# clocks sampled with nvidia-smi while the GPU is busy
# --------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="sg_clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "50", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = []
        if self.path and os.path.exists(self.path):
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9:
                        rows.append(parts)
            os.unlink(self.path)
        return summarize_clocks(rows)


def summarize_clocks(rows):
    if not rows:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = set()
    for r in rows:
        for name, val in zip(names, r[5:9]):
            if val.lower().startswith("active"):
                reasons.add(name)
    power = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "reasons": sorted(reasons),
            "power_w_max": max(power) if power else None,
            "samples": len(rows)}


# --------------------------------------------------------------------------
# roofline helpers
# --------------------------------------------------------------------------
def touched_bytes(r: int, elem: int, granule: int) -> int:
    """Bytes of the aligned granules (32-byte sectors or 128-byte lines) of the
    row-major n x n grid that hold at least one gasket cell.  A granule of
    2^g elements on row y starting at column x0 (a multiple of 2^g) holds one
    iff (x0 >> g) & (y >> g) == 0, so there are 2^g * 3^(r-g) of them."""
    per = granule // elem
    g = per.bit_length() - 1
    if g >= r:
        return (1 << r) * (1 << r) * elem if g > r else granule * (1 << r)
    return (1 << g) * 3 ** (r - g) * granule


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def recorded_traffic(kernel_key: str, unit: str):
    """DRAM bytes (read + write) per launch of this kernel from the committed
    ncu summary profiles/traffic.txt (lines: key, source digest of the
    kernel's translation unit, bytes), or None when that unit's sources or
    flags changed since the capture."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    try:
        from paper_1706_04552_gb300 import build as sg_build
        digest = sg_build.unit_digest(unit)
        with open(path) as f:
            for line in f:
                parts = line.split()
                if len(parts) == 3 and not line.startswith("#") and parts[0] == kernel_key:
                    return int(parts[2]) if parts[1] == digest else None
    except Exception:
        pass
    return None


# --------------------------------------------------------------------------
# timing on the device
# --------------------------------------------------------------------------
def balanced_chunks(total: int, k: int) -> list[int]:
    """Split `total` steps into the fewest launches of at most k steps, as
    even as they go (100 steps at k = 8: nine launches of 8 and four of 7).
    A launch of few steps costs nearly as much as one of k (both make one
    pass over the grid), so a short remainder launch is avoided."""
    n = -(-total // k)
    base, extra = divmod(total, n)
    return [base + 1] * extra + [base] * (n - extra)


def time_launches(fn, steps: int, stream):
    """Run fn() `steps` times on `stream`; CUDA events around the whole run
    and around every launch.  Returns (total ms, list of per-launch ms)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    t1.record(stream)
    t1.synchronize()
    return t0.elapsed_time(t1), [a.elapsed_time(b) for a, b in ev]


def soak(fn, seconds: float, stream):
    """Keep the GPU busy with fn() for about `seconds` (untimed)."""
    import torch
    t_end = time.time() + seconds
    while time.time() < t_end:
        for _ in range(50):
            fn()
        stream.synchronize()


# --------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------
def run_ours(args, grp: Group):
    import torch
    import paper_1706_04552_gb300 as sg
    from paper_1706_04552_gb300 import workloads

    sg.lib()                                   # fails loudly without libsg.so
    dev = torch.device("cuda", grp.local)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    if args.quick and args.l2_fetch:
        torch.zeros(1, device=dev)             # the context exists
        out = _with_l2_fetch_granularity(args.l2_fetch, lambda: run_ours_body(
            args, grp, sg, torch, dev, stream))
        return out
    return run_ours_body(args, grp, sg, torch, dev, stream)


def run_ours_body(args, grp, sg, torch, dev, stream):
    from paper_1706_04552_gb300 import workloads
    if args.quick and args.workload == "batch_ca_fused":
        return run_batch_quick(args, sg, torch, dev, stream)
    if args.quick and args.workload == "serve_fused":
        return run_serve_quick(args)
    if args.quick and args.workload != "write":
        return run_stencil_quick(args, sg, torch, dev, stream)
    w = dict(workloads.WRITE_HEADLINE)
    if args.rho:
        w["rho"] = args.rho
    if args.map:
        w["map"] = args.map
    if args.order:
        w["order"] = args.order
    if args.store:
        w["store"] = args.store
    if args.value:
        w["value"] = args.value
    if args.quick and args.level:
        w["r"] = args.level
    if args.quick and args.dtype == "f32":
        w["rho"] = args.rho or w["f32_rho"]
        w["store"] = args.store or w["f32_store"]
    r, n = w["r"], 1 << w["r"]
    cells = 3 ** r
    grid = torch.zeros(n * n, dtype=torch.uint8 if args.dtype == "u8" or not args.quick
                       else torch.float32, device=dev)

    def step():
        sg.map_write(grid, r, w["rho"], w["map"], w["value"], w["seed"], stream,
                     order=w["order"], store=w["store"])

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(torch.cuda.current_device())
    if not args.quick:
        sampler.start()
        soak(step, 1.0, stream)               # clocks settle, sampler sees load
    grp.barrier()
    torch.cuda.synchronize(dev)
    total_ms, per_launch = time_launches(step, args.steps, stream)
    torch.cuda.synchronize(dev)
    grp.barrier()
    clocks = sampler.stop()
    total_ms = grp.max(total_ms)

    ms_per_step = total_ms / args.steps
    value = grp.world * cells * args.steps / (total_ms / 1e3) / 1e9
    launch_ms = statistics.mean(per_launch)
    peak, peak_kind = measured_peak()
    elem = 4 if grid.dtype == torch.float32 else 1
    line_bytes = touched_bytes(r, elem, 128)
    sector_bytes = touched_bytes(r, elem, 32)
    achieved = line_bytes / (launch_ms / 1e3) / 1e9
    launched, useful = sg.launch_stats(r, w["rho"], w["map"])
    kernel_key = f"write_{w['map']}_{w['store']}_{w['order']}_r{r}_u8_rho{w['rho']}"
    roofline = {
        "bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
        "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
        # the same against the nominal HBM3e figure (about 8 TB/s)
        "peak_nominal": NOMINAL_HBM_GBS, "frac_nominal": round(achieved / NOMINAL_HBM_GBS, 4),
        "traffic": recorded_traffic(kernel_key, "sg_write_u8.cu"),
        "algorithmic_bytes_per_launch": line_bytes,
        "algorithmic_bytes": "touched 128-byte lines: 2^7 * 3^9 lines of 128 B",
        "sector_bytes_per_launch": sector_bytes,
        "achieved_sector_gbs": round(sector_bytes / (launch_ms / 1e3) / 1e9, 1),
        # the same against the 32-byte sectors the pass must write (stricter)
        "frac_sector": round(sector_bytes / (launch_ms / 1e3) / 1e9 / peak, 4),
        "launch_ms_mean": round(launch_ms, 5),
        "launch_ms_min": round(min(per_launch), 5),
        "kernel": kernel_key,
    }
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT,
        "n_gpus": grp.world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_per_step, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {
            "workload": (f"map-and-write, level {r} gasket in a {n}x{n} uint8 grid, "
                         f"hash(x,y) seed {w['seed']}, map {w['map']}, rho {w['rho']}, "
                         f"{w['order']} order, {w['store']} stores"),
            "r": r, "n": n, "rho": w["rho"], "map": w["map"], "order": w["order"],
            "store": w["store"], "value": w["value"],
            "seed": w["seed"], "cells_per_step": cells,
            "l2": "inputs larger than L2 (4.3 GB grid; 181 MB touched sectors > 129 MB L2)",
            "parallelism": "replicas" if grp.world > 1 else "single GPU",
        },
        "roofline": roofline,
        "threads": {"launched_slots": launched, "useful_cells": useful},
        "clocks": clocks,
        "gpu_launches": args.steps,
    }

    if roofline["traffic"]:
        # ncu DRAM bytes against the touched sectors: above 1 means bytes the
        # method does not need (here whole 64-byte tile rows)
        roofline["traffic_ratio"] = round(roofline["traffic"] / sector_bytes, 3)
    if args.quick:
        return out
    if grp.rank == 0 and not args.no_extras:
        out["compare"] = compare_workloads(sg, torch, dev, stream, w, grid, launch_ms)
        out["compare"]["level_sweep"] = level_sweep(sg, torch, dev, w)
        # each map at its own best (rho, store path) per level and element type
        ws = write_sweep(args)
        out["compare"]["write_sweep_best"] = {"protocol": ws["protocol"],
                                              "best_per_level": ws["best_per_level"]}
        out["compare"]["batched_ca"] = batched_workload(sg, torch, dev, stream)
        out["serving"] = serving_workload()
    del grid
    torch.cuda.empty_cache()
    copy = measure_e2e(sg, torch, dev, stream, w, grp, min(args.steps, 4))
    mapped = measure_e2e_mapped(sg, torch, dev, stream, w, grp, 20, "merge")
    mapped_staged = measure_e2e_mapped(sg, torch, dev, stream, w, grp, 20, "staged")
    mapped_fill = measure_e2e_mapped(sg, torch, dev, stream, w, grp, 20, "fill")
    mapped_sector = measure_e2e_mapped(sg, torch, dev, stream, w, grp, 20, "sector")
    # the headline end-to-end path reads the grid's inputs and writes the
    # result over the link, correct for any grid content (32-byte merge, the
    # library default; staged chunks beside it); the write-only paths (the
    # grid 0 off the gasket, as here) read nothing and are reported beside it
    best = max((mapped, mapped_staged, copy), key=lambda e: e["value"])
    out["e2e"] = dict(best)
    link = link_rates(torch, dev, grp)
    if link:
        # the link's own copy rates: the preserving path moves the touched
        # sectors both ways at once, the write-only paths one way
        out["e2e"]["link"] = link
        sec = touched_bytes(w["r"], 1, 32)
        out["e2e"]["link_frac"] = round(
            sec / (best["ms_per_step"] / 1e3) / 1e9 / link["bidir_each_GBs"], 3) \
            if best is not copy else None
        mapped_sector["link_frac"] = round(
            sec / (mapped_sector["ms_per_step"] / 1e3) / 1e9 / link["d2h_GBs"], 3)
    compact_mapped = measure_e2e_compact_mapped(sg, torch, dev, stream, w, grp, 20)
    out["e2e_paths"] = {"mapped": mapped, "mapped_staged": mapped_staged,
                        "mapped_fill": mapped_fill, "mapped_sector": mapped_sector,
                        "copy": copy, "compact_mapped": compact_mapped}
    if grp.rank == 0 and grp.world == 1 and not args.no_cpu:
        out["cpu_baseline"] = cpu_baseline(w)
        try:
            out["cpu_baseline_all_cores"] = cpu_baseline_all_cores(w)
        except Exception as e:                      # reported, never fatal
            out["cpu_baseline_all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"}
    return out


def run_batch_quick(args, sg, torch, dev, stream):
    """K launches of 16 fused CA steps of the batch of 64 gaskets (levels
    8..14, or 8..--level, rho 64, no autotuning), the batched serving
    kernel; for ncu."""
    from paper_1706_04552_gb300 import inputs, workloads
    w = workloads.BATCH
    hi = args.level if args.level else w["level_hi"]
    levels = inputs.batch_levels(w["count"], w["level_lo"], hi, w["level_seed"])
    a, b = [], []
    for i, r in enumerate(levels):
        idx, vals = inputs.ca_seed_sparse(r, w["ca_p"], inputs.instance_seed(w["ca_seed"], i))
        t = torch.zeros(1 << (2 * r), dtype=torch.uint8, device=dev)
        t[torch.from_numpy(idx).to(dev)] = torch.from_numpy(vals).to(dev)
        a.append(t)
        b.append(torch.zeros_like(t))
    k = w["fuse"]
    batch = sg.CABatch(levels, a, b, rho=64, stream=stream)
    par = [0]

    def step():
        batch.steps(k, par[0], stream)
        par[0] ^= 1
    for _ in range(max(3, args.warmup)):
        step()
    total_ms, per = time_launches(step, args.steps, stream)
    cells = sum(3 ** r for r in levels)
    return {"workload": f"{args.workload}, {len(levels)} gaskets of levels "
                        f"{w['level_lo']}..{hi}, rho 64, {k} steps per launch",
            "unit": UNIT, "value": round(cells * k / (total_ms / args.steps / 1e3) / 1e9, 3),
            "launch_ms_mean": round(statistics.mean(per), 5), "steps": args.steps}


def run_serve_quick(args):
    """The serving configuration with fused batches on the native core: one
    0.25 s trace at 160,000 req/s (--steps traces, after --warmup traces at
    2000 req/s); for the launch list of a serving run."""
    import dataclasses
    from paper_1706_04552_gb300.serve import ServeConfig, Server, make_trace, summarize
    base = ServeConfig(fuse=16)
    server = Server(base)
    warm = dataclasses.replace(base, rate=2000.0, duration=0.05)
    for _ in range(max(1, args.warmup)):
        server.run(make_trace(warm))
    cfg = dataclasses.replace(base, rate=160000.0, duration=0.25)
    out = []
    for _ in range(max(1, args.steps)):
        out.append(summarize(server.run(make_trace(cfg)), cfg))
    return {"workload": "serve_fused, 500 gaskets, 160000 req/s for 0.25 s, native core",
            "runs": out}


def run_stencil_quick(args, sg, torch, dev, stream):
    """K launches of the level-15 (or --level) CA or diffusion step, or of
    its fused form (k steps per launch), lambda map; for ncu."""
    from paper_1706_04552_gb300 import inputs, workloads
    s = workloads.STENCILS
    r = args.level if args.level else max(s["levels"])
    n = 1 << r
    kind, fused = args.workload.split("_")[0], args.workload.endswith("_fused")
    compact = "_compact" in args.workload
    if kind == "ca":
        idx, vals = inputs.ca_seed_sparse(r, s["ca_p"], s["ca_seed"])
        dt = torch.uint8
        rho, k = (s["ca_fuse_rho"], s["ca_fuse"]) if fused else (s["ca_rho"], 1)
    else:
        idx, vals = inputs.uniform_sparse(r, s["diff_seed"])
        dt = torch.float32
        rho, k = (s["diff_fuse_rho"], s["diff_fuse"]) if fused else (s["diff_rho"], 1)
    a = torch.zeros(n * n, dtype=dt, device=dev)
    a[torch.from_numpy(idx).to(dev)] = torch.from_numpy(vals).to(dev)
    if compact:
        rho = workloads.COMPACT["rho"]
        a = sg.compact_pack(a, torch.empty(3 ** r, dtype=dt, device=dev), r, rho, stream=stream)
    bufs = [a, torch.zeros_like(a)]

    def step():
        if compact and kind == "ca" and fused:
            sg.compact_ca_steps(bufs[0], bufs[1], r, rho, k, stream=stream)
        elif compact and kind == "ca":
            sg.compact_ca_step(bufs[0], bufs[1], r, rho, stream=stream)
        elif compact:
            sg.compact_diffuse_step(bufs[0], bufs[1], r, rho, s["alpha"], stream=stream)
        elif kind == "ca" and k == 1:
            sg.ca_step(bufs[0], bufs[1], r, rho, "lambda", stream, staging=args.staging)
        elif kind == "ca":
            sg.ca_steps(bufs[0], bufs[1], r, rho, k, "lambda", stream)
        elif k == 1:
            sg.diffuse_step(bufs[0], bufs[1], r, rho, s["alpha"], "lambda", stream,
                            staging=args.staging)
        else:
            sg.diffuse_steps(bufs[0], bufs[1], r, rho, k, s["alpha"], "lambda", stream)
        bufs.reverse()
    for _ in range(max(3, args.warmup)):
        step()
    total_ms, per = time_launches(step, args.steps, stream)
    return {"workload": f"{args.workload}, level {r}, rho {rho}, {k} step(s) per launch, "
                        + ("compact layout" if compact else "lambda")
                        + (f", {args.staging} staging" if args.staging else ""),
            "unit": UNIT, "value": round(3 ** r * k / (total_ms / args.steps / 1e3) / 1e9, 3),
            "launch_ms_mean": round(statistics.mean(per), 5), "steps": args.steps}


def batched_workload(sg, torch, dev, stream):
    """64 gaskets of levels 8..14: 64 CA steps as (a) one launch per gasket
    per step, eager and captured in a CUDA graph, and (b) one batched launch
    per step over the prefix-summed work list, eager and as a CUDA graph
    (autotuned rho / order / CTAs per SM)."""
    from paper_1706_04552_gb300 import inputs, workloads
    w = workloads.BATCH
    levels = inputs.batch_levels(w["count"], w["level_lo"], w["level_hi"], w["level_seed"])
    a, b = [], []
    for i, r in enumerate(levels):
        idx, vals = inputs.ca_seed_sparse(r, w["ca_p"], inputs.instance_seed(w["ca_seed"], i))
        t = torch.zeros(1 << (2 * r), dtype=torch.uint8, device=dev)
        t[torch.from_numpy(idx).to(dev)] = torch.from_numpy(vals).to(dev)
        a.append(t)
        b.append(torch.zeros_like(t))
    steps = w["steps"]
    cells = sum(3 ** r for r in levels) * steps
    batch = sg.CABatch(levels, a, b, autotune=w["autotune_steps"], stream=stream)
    opts = batch.opts
    order = "interleaved" if opts.order == 1 else "rowmajor"
    res = {"gaskets": len(levels), "levels": levels, "steps": steps,
           "profile": "profiles/batch_ca_bits_l8to12_rho64_k16.md",
           "cells_per_step": sum(3 ** r for r in levels),
           "tuned": {"rho": batch.rho, "order": order, "ctas_per_sm": opts.ctas_per_sm}}

    def per_instance():
        for k in range(steps):
            for i, r in enumerate(levels):
                src, dst = (a[i], b[i]) if k % 2 == 0 else (b[i], a[i])
                sg.ca_step(src, dst, r, batch.rho, "lambda", stream, order=order)

    def batched():
        for k in range(steps):
            batch.step(k & 1, stream)

    g = batch.graph(steps, 0)
    torch_graph = torch.cuda.CUDAGraph()
    per_instance()                                 # warm-up (and occupancy caches)
    torch.cuda.synchronize(dev)
    with torch.cuda.graph(torch_graph, stream=torch.cuda.Stream(dev)):
        s2 = torch.cuda.current_stream(dev)
        for k in range(steps):
            for i, r in enumerate(levels):
                src, dst = (a[i], b[i]) if k % 2 == 0 else (b[i], a[i])
                sg.ca_step(src, dst, r, batch.rho, "lambda", s2, order=order)
    torch.cuda.synchronize(dev)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize(dev)
        ms, _ = time_launches(fn, reps, stream)
        return ms / reps

    t_pi = timed(per_instance)
    t_pig = timed(lambda: torch_graph.replay())
    t_b = timed(batched)
    t_bg = timed(lambda: g.launch(stream))
    g.close()
    # the same 64 steps as launches of `fuse` fused steps (bit-sliced tiles),
    # autotuned for that launch shape, captured in one graph
    fb = sg.CABatch(levels, a, b, autotune=w["autotune_steps"], stream=stream, fuse=w["fuse"])
    gf = fb.graph(steps, 0, fuse=w["fuse"])
    t_fg = timed(lambda: gf.launch(stream))
    gf.close()
    fo = fb.opts
    res["batched_fused_graph"] = {
        "ms": round(t_fg, 3), "GCells_s": _rate(cells, t_fg), "steps_per_launch": w["fuse"],
        "launches": -(-steps // w["fuse"]),
        "tuned": {"rho": fb.rho, "order": "interleaved" if fo.order == 1 else "rowmajor",
                  "ctas_per_sm": fo.ctas_per_sm},
        "speedup_over_batched_graph": round(t_bg / t_fg, 3),
        "speedup_over_per_gasket_graph": round(t_pig / t_fg, 3)}
    del fb
    res.update({
        "per_gasket_eager": {"ms": round(t_pi, 3), "GCells_s": _rate(cells, t_pi),
                             "launches": steps * len(levels)},
        "per_gasket_graph": {"ms": round(t_pig, 3), "GCells_s": _rate(cells, t_pig),
                             "launches": steps * len(levels)},
        "batched_eager": {"ms": round(t_b, 3), "GCells_s": _rate(cells, t_b), "launches": steps},
        "batched_graph": {"ms": round(t_bg, 3), "GCells_s": _rate(cells, t_bg), "launches": steps},
        "speedup_batched_graph_over_per_gasket_eager": round(t_pi / t_bg, 3),
        "speedup_batched_graph_over_per_gasket_graph": round(t_pig / t_bg, 3),
    })
    del a, b, batch
    torch.cuda.empty_cache()
    return res


def level_sweep(sg, torch, dev, w):
    """lambda vs bounding box at every level 8..16 (uint8, hash values, the
    headline's intra-tile map, walking order and stores, rho = min(64, n)):
    GPU time per launch from CUDA-graph replays of 20 back-to-back launches,
    so host launch overhead does not mask the small levels."""
    out = {}
    for r in range(8, 17):
        n = 1 << r
        rho = min(64, n)
        g = torch.zeros(n * n, dtype=torch.uint8, device=dev)
        row = {}
        for name, mapk in (("lambda", w["map"]), ("bbox", "bbox")):
            cap = torch.cuda.Stream(dev)
            sg.map_write(g, r, rho, mapk, "hash", w["seed"], order=w["order"], store=w["store"])
            torch.cuda.synchronize(dev)
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=cap):
                for _ in range(20):
                    sg.map_write(g, r, rho, mapk, "hash", w["seed"], torch.cuda.current_stream(dev),
                                 order=w["order"], store=w["store"])
            graph.replay()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s = torch.cuda.current_stream(dev)
            e0.record(s)
            for _ in range(5):
                graph.replay()
            e1.record(s)
            e1.synchronize()
            us = e0.elapsed_time(e1) * 1e3 / 100
            row[name + "_us"] = round(us, 2)
            del graph
        row["speedup"] = round(row["bbox_us"] / row["lambda_us"], 3)
        row["GCells_s_lambda"] = round(3 ** r / row["lambda_us"] / 1e3, 2)
        out[f"r{r}"] = row
        del g
        torch.cuda.empty_cache()
    return out


def paper_sweep(args):
    """The paper's write experiment (its Section IV): the mean time of writing
    a constant into every gasket cell of a zero n x n matrix, over levels
    0..16 and block sizes rho = 1, 2, ..., 32, for lambda and the bounding box.
    Each point is the mean of 100 sub-averages, each the mean of 10
    consecutive calls; the 10 calls are replayed from a CUDA graph so the time
    is the GPU's, not the host's launch overhead.  Both maps use the paper's
    kernel structure: a thread per slot of the rho x rho sub-box with its
    membership test and a per-cell store."""
    import math
    import torch
    import paper_1706_04552_gb300 as sg
    sg.lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    rows = []
    # written before every sub-average (outside its events) so that each one
    # starts with the grid out of L2, as a fresh series of calls would
    l2 = int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0)) or (129 << 20)
    flush = torch.empty(2 * l2, dtype=torch.uint8, device=dev)
    for r in range(0, 17):
        n = 1 << r
        g = torch.zeros(n * n, dtype=torch.uint8, device=dev)
        for rho in (1, 2, 4, 8, 16, 32):
            if rho > n:
                continue
            point = {"r": r, "rho": rho}
            for name, mapk in (("lambda", "lambda"), ("bbox", "bbox")):
                cap = torch.cuda.Stream(dev)
                call = lambda st: sg.map_write(g, r, rho, mapk, "const", 1, st, order="rowmajor",
                                               store="scatter")
                call(torch.cuda.current_stream(dev))
                torch.cuda.synchronize(dev)
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph, stream=cap):
                    for _ in range(10):
                        call(torch.cuda.current_stream(dev))
                graph.replay()
                torch.cuda.synchronize(dev)
                # a few probe replays decide how many sub-averages fit ~2 s
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s = torch.cuda.current_stream(dev)
                e0.record(s)
                graph.replay()
                e1.record(s)
                e1.synchronize()
                probe_ms = e0.elapsed_time(e1)
                subs = 100 if probe_ms * 100 < 2000 else max(10, int(2000 / max(probe_ms, 1e-3)))
                vals = []
                for k in range(subs):
                    flush.fill_(k & 0xFF)
                    e0.record(s)
                    graph.replay()
                    e1.record(s)
                    e1.synchronize()
                    vals.append(e0.elapsed_time(e1) * 1e3 / 10)
                mean = statistics.mean(vals)
                se = statistics.stdev(vals) / math.sqrt(len(vals)) if len(vals) > 1 else 0.0
                point[name + "_us"] = round(mean, 3)
                point[name + "_se_pct"] = round(100 * se / mean, 3)
                point[name + "_subaverages"] = subs
                del graph
            point["speedup"] = round(point["bbox_us"] / point["lambda_us"], 3)
            rows.append(point)
        del g
        torch.cuda.empty_cache()
    best = {}
    for r in range(0, 17):
        pts = [p for p in rows if p["r"] == r]
        bl = min(pts, key=lambda p: p["lambda_us"])
        bb = min(pts, key=lambda p: p["bbox_us"])
        best[f"r{r}"] = {"lambda_rho": bl["rho"], "lambda_us": bl["lambda_us"],
                         "bbox_rho": bb["rho"], "bbox_us": bb["bbox_us"],
                         "speedup_best_vs_best": round(bb["bbox_us"] / bl["lambda_us"], 3)}
    return {"experiment": "paper Section IV: constant write into the gasket of a zero "
                          "uint8 matrix, lambda (bounding sub-boxes) vs bounding box",
            "protocol": "mean of 100 sub-averages of 10 consecutive calls (CUDA-graph "
                        "replay); fewer sub-averages where 100 would exceed ~2 s; L2 "
                        "flushed (a 2x L2 write) before every sub-average; grids of "
                        "r <= 13 (<= 64 MB) stay L2-resident within a sub-average",
            "points": rows, "best_per_level": best}


SWEEP_LAUNCHES = 50


def write_sweep(args):
    """The map-and-write sweep over levels 8..16, uint8 and float32 grids,
    rho = 8, 16, 32, 64, lambda (the headline's intra-tile map and walking
    order) against the bounding box, hash values seed 1, each with every
    store path the tile rows allow (per-cell stores; whole-tile fill stores
    where a tile row holds at least 16 bytes; whole-sector stores where it
    holds at least 32).  Each point: GPU time per launch from CUDA-graph
    replays of 50 launches (the L2 flushed before each timed replay),
    GCells/s, launched against useful cell slots, and touched 128-byte lines
    per second; each map's best point per level is compared."""
    import torch
    import paper_1706_04552_gb300 as sg
    from paper_1706_04552_gb300 import workloads
    sg.lib()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    sw, hw = workloads.WRITE_SWEEP, workloads.WRITE_HEADLINE
    l2 = int(getattr(torch.cuda.get_device_properties(dev), "L2_cache_size", 0)) or (129 << 20)
    flush = torch.empty(2 * l2, dtype=torch.uint8, device=dev)
    peak, peak_kind = measured_peak()
    rows = []
    for dtype, elem, tdt in (("u8", 1, torch.uint8), ("f32", 4, torch.float32)):
        for r in sw["levels"]:
            n = 1 << r
            g = torch.zeros(n * n, dtype=tdt, device=dev)
            lines = touched_bytes(r, elem, 128)
            for rho in sw["rhos"]:
                if rho > n:
                    continue
                # every store path the tile rows allow, for both maps: each
                # map is then compared at its best (rho, store)
                stores = ["scatter"] + (["fill"] if rho * elem >= 16 else []) + \
                         (["sector"] if rho * elem >= 32 else [])
                for store, (name, mapk) in ((st_, m_) for st_ in stores for m_ in (
                        ("lambda", hw["map"]), ("bbox", "bbox"))):
                    cap = torch.cuda.Stream(dev)
                    call = lambda st: sg.map_write(g, r, rho, mapk, "hash", hw["seed"], st,
                                                   order=hw["order"], store=store)
                    call(torch.cuda.current_stream(dev))
                    torch.cuda.synchronize(dev)
                    graph = torch.cuda.CUDAGraph()
                    with torch.cuda.graph(graph, stream=cap):
                        for _ in range(SWEEP_LAUNCHES):
                            call(torch.cuda.current_stream(dev))
                    graph.replay()
                    torch.cuda.synchronize(dev)
                    st = torch.cuda.current_stream(dev)
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    vals = []
                    for k in range(5):
                        flush.fill_(k & 0xFF)
                        e0.record(st)
                        graph.replay()
                        e1.record(st)
                        e1.synchronize()
                        vals.append(e0.elapsed_time(e1) * 1e3 / SWEEP_LAUNCHES)
                    us = statistics.median(vals)
                    launched, useful = sg.launch_stats(r, rho, mapk)
                    rows.append({"dtype": dtype, "r": r, "rho": rho, "map": mapk, "store": store,
                                 "us": round(us, 2), "GCells_s": round(3 ** r / us / 1e3, 2),
                                 "launched_slots": launched, "useful_cells": useful,
                                 "line_GBps": round(lines / us / 1e3, 1),
                                 "frac": round(lines / us / 1e3 / peak, 3)})
                    del graph
            del g
            torch.cuda.empty_cache()
    best = {}
    for dtype in ("u8", "f32"):
        for r in sw["levels"]:
            pts = [p for p in rows if p["dtype"] == dtype and p["r"] == r]
            bl = min((p for p in pts if p["map"] != "bbox"), key=lambda p: p["us"])
            bb = min((p for p in pts if p["map"] == "bbox"), key=lambda p: p["us"])
            best[f"{dtype}_r{r}"] = {"lambda_rho": bl["rho"], "lambda_us": bl["us"],
                                     "lambda_GCells_s": bl["GCells_s"], "lambda_frac": bl["frac"],
                                     "bbox_rho": bb["rho"], "bbox_us": bb["us"],
                                     "speedup_best_vs_best": round(bb["us"] / bl["us"], 3)}
    return {"experiment": "map-and-write sweep: levels 8..16, uint8 and float32, rho 8..64, "
                          "lambda vs bounding box, hash values seed 1",
            "protocol": "median of 5 CUDA-graph replays of 50 launches, L2 flushed before each",
            "peak_GBps": peak, "peak_kind": peak_kind, "points": rows, "best_per_level": best}


SATURATION_RATES = (2000.0, 5000.0, 10000.0, 20000.0, 40000.0, 80000.0, 160000.0, 320000.0,
                    640000.0, 1280000.0, 2560000.0)
SATURATION_P99_MS = 5.0


def serving_workload():
    """Continuous batching of CA-step requests (Poisson arrivals, 500 resident
    gaskets of levels 6..15, 1-32 steps per request, 40 GB budget) in four
    modes: batched launches of one step and of up to 16 fused steps on the
    native scheduler core, the fused batches again with the scheduler in
    Python, and one launch per active gasket.  Each mode serves the configured
    2000 req/s for 2 s and then traces of 5000 to 2560000 req/s (4000 requests
    or 0.25 s, whichever is longer), stopping after the first rate it does not
    sustain.  A mode sustains an offered rate when it serves the trace at
    >= 95 % of the trace's own arrival rate, with p99 latency <= 5 ms and no
    failed request; `max_sustained_rps` is the highest such rate."""
    import dataclasses
    from paper_1706_04552_gb300.serve import ServeConfig, Server, make_trace, summarize
    modes = (("batched", "batched", 1, "native"), ("batched_fused16", "batched", 16, "native"),
             ("batched_fused16_python", "batched", 16, "python"),
             ("per_gasket", "per_gasket", 1, "python"))
    sat = {"p99_bound_ms": SATURATION_P99_MS, "rates_rps": list(SATURATION_RATES),
           "modes": {}}
    out = {}
    for name, mode, fuse, engine in modes:
        base = ServeConfig(mode=mode, fuse=fuse, engine=engine)
        server = Server(base)
        rows, best = [], None
        for rate in SATURATION_RATES:
            dur = base.duration if rate <= base.rate else max(0.25, 4000.0 / rate)
            cfg = dataclasses.replace(base, rate=rate, duration=dur)
            trace = make_trace(cfg)
            res = server.run(trace)
            s = summarize(res, cfg)
            arrival_rps = len(trace[0]) / dur
            s["served_fraction"] = round(s["throughput_rps"] / arrival_rps, 4)
            s["sustained"] = bool(s["served_fraction"] >= 0.95 and s["failed"] == 0
                                  and s["latency_ms_p99"] <= SATURATION_P99_MS)
            rows.append(s)
            if rate == base.rate:
                out.setdefault("offered_2000rps", {})[name] = s
            if not s["sustained"]:
                break
            best = rate
        sat["modes"][name] = {"max_sustained_rps": best, "points": rows}
        del server
    sat["profile"] = "profiles/serving_fused_launches.md"
    out["saturation"] = sat
    return out


def _rate(cells, ms):
    return round(cells / (ms / 1e3) / 1e9, 3)


def _memset_rate(torch, t, stream, reps=4, nbytes=None):
    """Write bandwidth of cuMemsetD8Async over a whole device tensor, or over
    its first `nbytes` bytes (the fastest way to write every byte of it):
    bytes / best event-timed call."""
    import ctypes
    try:
        cu = ctypes.CDLL("libcuda.so.1")
    except OSError as e:
        return {"unavailable": f"libcuda: {e}"}
    whole = nbytes is None
    nbytes = t.numel() * t.element_size() if whole else min(int(nbytes), t.numel() *
                                                              t.element_size())
    ms = []
    for i in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rc = cu.cuMemsetD8Async(ctypes.c_uint64(t.data_ptr()), ctypes.c_ubyte(i & 0xFF),
                                ctypes.c_size_t(nbytes), ctypes.c_void_p(stream.cuda_stream))
        e1.record(stream)
        e1.synchronize()
        if rc != 0:
            return {"unavailable": f"cuMemsetD8Async returned {rc}"}
        ms.append(e0.elapsed_time(e1))
    best = min(ms[1:])
    what = "the whole grid" if whole else "the grid's first bytes, contiguous"
    return {"bytes": nbytes, "ms": round(best, 4), "GBps": round(nbytes / (best / 1e3) / 1e9, 1),
            "how": f"cuMemsetD8Async over {what}, best of 4 after one warm-up"}


def _add_traffic(entry, key, unit, launch_us):
    """Attach the recorded ncu DRAM bytes of one launch (profiles/traffic.txt,
    while the unit's code still matches) and the DRAM rate they give at the
    measured launch time, as a fraction of the measured HBM peak."""
    t = recorded_traffic(key, unit)
    entry["traffic_bytes_per_launch"] = t
    if t:
        peak, kind = measured_peak()
        gbs = t / (launch_us / 1e6) / 1e9
        entry["dram_GBps"] = round(gbs, 1)
        entry["dram_frac"] = round(gbs / peak, 4)
        entry["dram_peak_kind"] = kind


def _time_leg(sg, grid, r, cfg, seed, stream, cells, sector_b, steps):
    f = lambda: sg.map_write(grid, r, cfg["rho"], cfg["map"], "hash", seed, stream,
                             order=cfg["order"], store=cfg["store"])
    for _ in range(3):
        f()
    ms, per = time_launches(f, steps, stream)
    return {"map": cfg["map"], "rho": cfg["rho"], "order": cfg["order"], "store": cfg["store"],
            "GCells_s": _rate(cells, ms / steps), "launch_ms": round(statistics.mean(per), 5),
            "sector_GBps": round(sector_b / (statistics.mean(per) / 1e3) / 1e9, 1)}


def _with_l2_fetch_granularity(nbytes, fn):
    """Run fn() with the current CUDA context's L2 fetch granularity limit
    (CU_LIMIT_MAX_L2_FETCH_GRANULARITY) set to nbytes, then put the previous
    value back.  The limit belongs to this process's context only."""
    import ctypes
    try:
        cu = ctypes.CDLL("libcuda.so.1")
    except OSError as e:
        return {"unavailable": f"libcuda: {e}"}
    limit = 0x05                       # CU_LIMIT_MAX_L2_FETCH_GRANULARITY
    old = ctypes.c_size_t(0)
    if cu.cuCtxGetLimit(ctypes.byref(old), limit) != 0:
        return {"unavailable": "cuCtxGetLimit failed"}
    if cu.cuCtxSetLimit(limit, ctypes.c_size_t(nbytes)) != 0:
        return {"unavailable": "cuCtxSetLimit failed"}
    try:
        out = fn()
    finally:
        cu.cuCtxSetLimit(limit, old)
    out["l2_fetch_granularity"] = {"set": nbytes, "default": old.value}
    return out


def compare_workloads(sg, torch, dev, stream, w, grid_u8, headline_launch_ms):
    """Short timings of the other configurations on the same GPU."""
    from paper_1706_04552_gb300 import inputs, workloads
    r, n = w["r"], 1 << w["r"]
    cells = 3 ** r
    res = {}
    # the bounding-box map on the same grid at its own best rho and the same
    # stores; the lambda pass with stores that keep arbitrary off-gasket
    # content; the paper's own intra-tile variant (bounding sub-boxes)
    from paper_1706_04552_gb300 import workloads as wl
    pv = wl.WRITE_PRESERVE
    sector_b = touched_bytes(r, 1, 32)
    legs = (("bbox_u8", "bbox", w["bbox_rho"], w["order"], w["bbox_store"], 20, "hash"),
            ("bbox_fill_u8", "bbox", w["bbox_rho"], w["order"], "fill", 20, "hash"),
            ("lambda_preserving_u8", pv["map"], pv["rho"], pv["order"], pv["store"], 200, "hash"),
            ("lambda_staged_u8", pv["map"], 32, "rowmajor", "staged", 200, "hash"),
            ("lambda_masked_u8", pv["map"], 64, w["order"], "masked", 100, "hash"),
            ("lambda_sector_u8", w["map"], 64, w["order"], "sector", 200, "hash"),
            ("lambda_subbox_u8", "lambda", w["rho"], w["order"], w["store"], 200, "hash"),
            # the store paths alone: a constant instead of the hash
            ("store_floor_fill_const_u8", w["map"], w["rho"], w["order"], w["store"], 200,
             "const"),
            ("store_floor_sector_const_u8", w["map"], 64, w["order"], "sector", 200, "const"))
    write_profile = "profiles/write_legs_r16.md"
    for name, mapk, rho, order, store, steps, vk in legs:
        f = lambda: sg.map_write(grid_u8, r, rho, mapk, vk, w["seed"], stream,
                                 order=order, store=store)
        for _ in range(3):
            f()
        grid_u8.zero_()
        ms, per = time_launches(f, steps, stream)
        res[name] = {"map": mapk, "rho": rho, "order": order, "store": store, "value": vk,
                     "GCells_s": _rate(cells, ms / steps),
                     "launch_ms": round(statistics.mean(per), 5),
                     "line_GBps": round(touched_bytes(r, 1, 128) /
                                        (statistics.mean(per) / 1e3) / 1e9, 1),
                     "sector_GBps": round(sector_b / (statistics.mean(per) / 1e3) / 1e9, 1),
                     "profile": write_profile}
    # the preserving merge pass with the L2 fetching 32 bytes per read miss
    # (a per-context limit of the CUDA driver, restored afterwards): DRAM then
    # reads the touched sectors only, instead of their whole 128-byte lines
    res["lambda_preserving_u8_l2fetch32"] = _with_l2_fetch_granularity(32, lambda: _time_leg(
        sg, grid_u8, r, pv, w["seed"], stream, cells, sector_b, 200))
    res["lambda_preserving_u8_l2fetch32"]["profile"] = write_profile
    # streaming write bandwidth of the same memory: the whole 4.3 GB grid
    # set by the driver's memset (every byte, in address order)
    res["stream_write_full_grid"] = _memset_rate(torch, grid_u8, stream)
    # the same number of bytes as the touched sectors, written contiguously:
    # what the pass would cost if its sectors were not scattered over the grid
    res["stream_write_sector_bytes_contiguous"] = _memset_rate(
        torch, grid_u8, stream, nbytes=touched_bytes(r, 1, 32))
    grid_u8.zero_()
    res["speedup_lambda_over_bbox"] = round(res["bbox_u8"]["launch_ms"] / headline_launch_ms, 3)
    # float32 grid (17.2 GB)
    g32 = torch.zeros(n * n, dtype=torch.float32, device=dev)
    f = lambda: sg.map_write(g32, r, w["f32_rho"], w["map"], "hash", w["seed"], stream,
                             order=w["order"], store=w["f32_store"])
    for _ in range(3):
        f()
    ms, per = time_launches(f, 100, stream)
    lb = touched_bytes(r, 4, 128)
    res["lambda_f32"] = {"map": w["map"], "rho": w["f32_rho"], "store": w["f32_store"],
                         "GCells_s": _rate(cells, ms / 100),
                         "launch_ms": round(statistics.mean(per), 5),
                         "line_GBps": round(lb / (statistics.mean(per) / 1e3) / 1e9, 1),
                         "profile": write_profile}
    del g32
    torch.cuda.empty_cache()
    # stencils at level 15
    s = workloads.STENCILS
    rs = max(s["levels"])
    ns, cs = 1 << rs, 3 ** rs
    idx, vals = inputs.ca_seed_sparse(rs, s["ca_p"], s["ca_seed"])
    tidx = torch.from_numpy(idx).to(dev)
    for mapk, rho in (("lambda", s["ca_rho"]), ("bbox", s["bbox_ca_rho"])):
        a = torch.zeros(ns * ns, dtype=torch.uint8, device=dev)
        a[tidx] = torch.from_numpy(vals).to(dev)
        b = torch.zeros_like(a)
        bufs = [a, b]

        def ca():
            sg.ca_step(bufs[0], bufs[1], rs, rho, mapk, stream)
            bufs.reverse()
        for _ in range(4):
            ca()
        steps = s["ca_steps"] if mapk == "lambda" else 32
        ms, per = time_launches(ca, steps, stream)
        lb = 2 * touched_bytes(rs, 1, 128)
        res[f"ca_r{rs}_{mapk}"] = {"rho": rho, "steps": steps,
                                   "GCells_s": _rate(cs, ms / steps),
                                   "launch_ms": round(statistics.mean(per), 5),
                                   "line_GBps": round(lb / (statistics.mean(per) / 1e3) / 1e9, 1)}
        if mapk == "lambda":
            _add_traffic(res[f"ca_r{rs}_{mapk}"], f"ca_r{rs}_lambda_rho{rho}", "sg_stencil.cu",
                         statistics.mean(per) * 1e3)
            res[f"ca_r{rs}_{mapk}"]["profile"] = ["profiles/ca_lambda_r15_rho64.md",
                                                  "profiles/stencil_staging_r15.md"]
        del a, b, bufs
    idx, vals = inputs.uniform_sparse(rs, s["diff_seed"])
    for mapk, rho in (("lambda", s["diff_rho"]), ("bbox", s["bbox_diff_rho"])):
        a = torch.zeros(ns * ns, dtype=torch.float32, device=dev)
        a[tidx] = torch.from_numpy(vals).to(dev)
        b = torch.zeros_like(a)
        bufs = [a, b]

        def df():
            sg.diffuse_step(bufs[0], bufs[1], rs, rho, s["alpha"], mapk, stream)
            bufs.reverse()
        for _ in range(4):
            df()
        steps = s["diff_steps"] if mapk == "lambda" else 20
        ms, per = time_launches(df, steps, stream)
        lb = 2 * touched_bytes(rs, 4, 128)
        res[f"diffusion_r{rs}_{mapk}"] = {"rho": rho, "steps": steps,
                                          "GCells_s": _rate(cs, ms / steps),
                                          "launch_ms": round(statistics.mean(per), 5),
                                          "line_GBps": round(lb / (statistics.mean(per) / 1e3) / 1e9, 1)}
        if mapk == "lambda":
            _add_traffic(res[f"diffusion_r{rs}_{mapk}"], f"diffusion_r{rs}_lambda_rho{rho}",
                         "sg_stencil.cu", statistics.mean(per) * 1e3)
            res[f"diffusion_r{rs}_{mapk}"]["profile"] = ["profiles/diffusion_lambda_r14_rho32.md",
                                                         "profiles/stencil_staging_r15.md"]
        del a, b, bufs
    torch.cuda.empty_cache()
    # the same step sequences with k steps fused per launch
    res.update(fused_stencils(sg, torch, dev, stream, rs, res))
    # the write pass and the step sequences on compact arrays
    res["compact"] = compact_layout(sg, torch, dev, stream, r, rs, res, headline_launch_ms)
    return res


def fused_stencils(sg, torch, dev, stream, r, single):
    """The level-r stencil sequences (256 CA steps, 100 diffusion steps) run
    as launches of k fused steps (sg_ca_steps / sg_diffuse_steps): rate in
    cell-steps per second and the ratio to the single-step launches."""
    from paper_1706_04552_gb300 import inputs, workloads
    s = workloads.STENCILS
    n, cells = 1 << r, 3 ** r
    out = {}
    for kind in ("ca", "diffusion"):
        if kind == "ca":
            idx, vals = inputs.ca_seed_sparse(r, s["ca_p"], s["ca_seed"])
            dt, total, k, rho = torch.uint8, s["ca_steps"], s["ca_fuse"], s["ca_fuse_rho"]
        else:
            idx, vals = inputs.uniform_sparse(r, s["diff_seed"])
            dt, total, k, rho = torch.float32, s["diff_steps"], s["diff_fuse"], s["diff_fuse_rho"]
        a = torch.zeros(n * n, dtype=dt, device=dev)
        a[torch.from_numpy(idx).to(dev)] = torch.from_numpy(vals).to(dev)
        bufs = [a, torch.zeros_like(a)]
        chunks = balanced_chunks(total, k)
        pos = [0]

        def launch():
            kk = chunks[pos[0] % len(chunks)]
            pos[0] += 1
            if kind == "ca":
                sg.ca_steps(bufs[0], bufs[1], r, rho, kk, "lambda", stream)
            else:
                sg.diffuse_steps(bufs[0], bufs[1], r, rho, kk, s["alpha"], "lambda", stream)
            bufs.reverse()
        for _ in range(len(chunks)):
            launch()                                   # warm-up: one whole sequence
        pos[0] = 0
        ms, per = time_launches(launch, len(chunks), stream)
        rate = cells * total / (ms / 1e3) / 1e9
        base = single.get(f"{kind}_r{r}_lambda", {}).get("GCells_s")
        out[f"{kind}_r{r}_fused"] = {
            "rho": rho, "steps": total, "steps_per_launch": k, "launches": len(chunks),
            "launch_steps": chunks,
            "us_per_step": round(ms * 1e3 / total, 2), "GCells_s": round(rate, 3),
            "speedup_vs_single_step": round(rate / base, 3) if base else None}
        # DRAM bytes of one launch of k steps, spread over its k steps
        _add_traffic(out[f"{kind}_r{r}_fused"], f"{kind}_fused_r{r}_rho{rho}_k{k}", "sg_fused.cu",
                     ms * 1e3 / total * k)
        out[f"{kind}_r{r}_fused"]["profile"] = ("profiles/ca_fused_bits_r15_rho64_k16.md"
                                                if kind == "ca" else
                                                "profiles/diffusion_warp_fused_r14_rho32_k8.md")
        del a, bufs
        torch.cuda.empty_cache()
    return out


def compact_layout(sg, torch, dev, stream, rw, rs, single, headline_launch_ms):
    """The level-rw write pass and the level-rs stencil sequences on compact
    arrays (only the 3^r gasket cells, tiles in launch order): rates, the
    bytes each form keeps on the device, and the ratio to the embedded runs.
    The compact stencil states start from the embedded seeds, packed."""
    from paper_1706_04552_gb300 import inputs, workloads
    c = workloads.COMPACT
    s = workloads.STENCILS
    rho, order = c["rho"], c["order"]
    out = {"rho": rho, "order": order}
    cw = 3 ** rw
    buf = torch.empty(cw, dtype=torch.uint8, device=dev)
    f = lambda: sg.compact_map_write(buf, rw, rho, "hash", 1, order=order, stream=stream)
    for _ in range(3):
        f()
    ms, per = time_launches(f, 200, stream)
    out[f"write_u8_r{rw}"] = {
        "GCells_s": _rate(cw, ms / 200), "launch_ms": round(statistics.mean(per), 5),
        "bytes_on_device": cw, "embedded_bytes_on_device": 1 << (2 * rw),
        "speedup_vs_embedded_fill": round(headline_launch_ms / statistics.mean(per), 3)}
    del buf
    n, cs = 1 << rs, 3 ** rs
    for kind in ("ca", "diffusion"):
        if kind == "ca":
            idx, vals = inputs.ca_seed_sparse(rs, s["ca_p"], s["ca_seed"])
            dt, total, elem = torch.uint8, s["ca_steps"], 1
        else:
            idx, vals = inputs.uniform_sparse(rs, s["diff_seed"])
            dt, total, elem = torch.float32, s["diff_steps"], 4
        g = torch.zeros(n * n, dtype=dt, device=dev)
        g[torch.from_numpy(idx).to(dev)] = torch.from_numpy(vals).to(dev)
        a = sg.compact_pack(g, torch.empty(cs, dtype=dt, device=dev), rs, rho, order=order,
                            stream=stream)
        del g
        bufs = [a, torch.empty_like(a)]

        def step():
            if kind == "ca":
                sg.compact_ca_step(bufs[0], bufs[1], rs, rho, order=order, stream=stream)
            else:
                sg.compact_diffuse_step(bufs[0], bufs[1], rs, rho, s["alpha"], order=order,
                                        stream=stream)
            bufs.reverse()
        for _ in range(4):
            step()
        ms, per = time_launches(step, total, stream)
        rate = cs * total / (ms / 1e3) / 1e9
        one = single.get(f"{kind}_r{rs}_lambda", {}).get("GCells_s")
        fused = single.get(f"{kind}_r{rs}_fused", {}).get("GCells_s")
        if kind == "ca":
            # the same sequence as launches of k fused steps
            k = s["ca_fuse"]
            chunks = balanced_chunks(total, k)
            pos = [0]

            def launch():
                sg.compact_ca_steps(bufs[0], bufs[1], rs, rho, chunks[pos[0] % len(chunks)],
                                    order=order, stream=stream)
                pos[0] += 1
                bufs.reverse()
            for _ in range(len(chunks)):
                launch()
            pos[0] = 0
            fms, _ = time_launches(launch, len(chunks), stream)
            frate = cs * total / (fms / 1e3) / 1e9
            out[f"ca_r{rs}_fused"] = {
                "steps": total, "steps_per_launch": k, "launches": len(chunks),
                "us_per_step": round(fms * 1e3 / total, 2), "GCells_s": round(frate, 3),
                "speedup_vs_embedded_fused": round(frate / fused, 3) if fused else None}
        out[f"{kind}_r{rs}"] = {
            "steps": total, "us_per_step": round(ms * 1e3 / total, 2),
            "GCells_s": round(rate, 3),
            # read + write of every element: both buffers fit in L2 for the CA
            "state_bytes": 2 * cs * elem, "embedded_state_bytes": 2 * n * n * elem,
            "speedup_vs_single_step": round(rate / one, 3) if one else None,
            "speedup_vs_fused": round(rate / fused, 3) if fused else None}
        del a, bufs
        torch.cuda.empty_cache()
    return out


def link_rates(torch, dev, grp, nbytes=1 << 31):
    """The host link's copy rates with the copy engines, pinned host memory
    <-> device memory, 2 GB sequential: host to device, device to host, and
    both at once on two streams (each direction's rate), on this rank's GPU.
    The denominators of the mapped paths' link fractions; None when the
    memory is not there."""
    try:
        h = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        h2 = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
        d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        d2 = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    except (RuntimeError, MemoryError):
        return None
    s1, s2 = torch.cuda.Stream(dev), torch.cuda.Stream(dev)

    def best_ms(fn, reps=4):
        fn()
        torch.cuda.synchronize(dev)
        out = []
        for _ in range(reps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            out.append(a.elapsed_time(b))
        return min(out)

    def bidir():
        cur = torch.cuda.current_stream(dev)
        s1.wait_stream(cur)
        s2.wait_stream(cur)
        with torch.cuda.stream(s1):
            d.copy_(h, non_blocking=True)
        with torch.cuda.stream(s2):
            h2.copy_(d2, non_blocking=True)
        cur.wait_stream(s1)
        cur.wait_stream(s2)

    res = {"h2d_GBs": nbytes / best_ms(lambda: d.copy_(h, non_blocking=True)) / 1e6,
           "d2h_GBs": nbytes / best_ms(lambda: h.copy_(d, non_blocking=True)) / 1e6,
           "bidir_each_GBs": nbytes / best_ms(bidir) / 1e6}
    del h, h2, d, d2
    torch.cuda.empty_cache()
    res = {k: round(v, 1) for k, v in res.items()}
    res["how"] = "cudaMemcpyAsync of 2 GB, pinned host <-> device, best of 4"
    return res


def measure_e2e_mapped(sg, torch, dev, stream, w, grp, steps, store="merge"):
    """The same metric through the public API with the grid kept in pinned
    host memory and written in place (sg_map_write_mapped): the kernel reads
    and writes the touched chunks of the host grid over the host link
    (NVLink-C2C); the preserving stores (staged 16-byte chunks, 32-byte merge)
    keep every other byte.
    Each step ends with the stream synchronised, the result in host memory."""
    from paper_1706_04552_gb300 import workloads
    r, n = w["r"], 1 << w["r"]
    m = workloads.WRITE_MAPPED
    host = torch.zeros(n * n, dtype=torch.uint8, pin_memory=True)

    def step():
        sg.map_write_mapped(host, r, m["rho"], m["map"], w["value"], w["seed"], stream,
                            order=m["order"], store=store)

    step()
    torch.cuda.synchronize(dev)
    grp.barrier()
    ms, _ = time_launches(step, steps, stream)
    ms = grp.max(ms)
    del host
    sector = touched_bytes(r, 1, 32)
    preserving = store in ("staged", "merge")
    reads = sector if preserving else 0
    how = ("the touched 32-byte sectors read and written back" if preserving else
           "the touched 32-byte sectors written whole, nothing read (the grid is 0 off "
           "the gasket)")
    return {"value": round(grp.world * 3 ** r * steps / (ms / 1e3) / 1e9, 4), "unit": UNIT,
            "h2d_bytes_per_step": reads, "d2h_bytes_per_step": sector,
            "steps": steps, "ms_per_step": round(ms / steps, 3),
            "path": (f"grid in pinned host memory, written in place by the kernel over the "
                     f"host link ({m['map']}, rho {m['rho']}, {m['order']}, {store} "
                     f"stores); bytes per step = {how}")}


def measure_e2e_compact_mapped(sg, torch, dev, stream, w, grp, steps):
    """The write pass in the compact layout (the 3^r gasket cells, tiles in
    launch order) written straight into pinned host memory over the host link
    (sg_compact_map_write_mapped): one contiguous run of whole sectors per
    pass, nothing read.  A different storage of the same cells and values as
    the embedded grid."""
    from paper_1706_04552_gb300 import workloads
    r = w["r"]
    rho = workloads.COMPACT["rho"]
    host = torch.zeros(3 ** r, dtype=torch.uint8, pin_memory=True)

    def step():
        sg.compact_map_write_mapped(host, r, rho, w["value"], w["seed"],
                                    order=workloads.COMPACT["order"], stream=stream)

    step()
    torch.cuda.synchronize(dev)
    grp.barrier()
    ms, _ = time_launches(step, steps, stream)
    ms = grp.max(ms)
    del host
    return {"value": round(grp.world * 3 ** r * steps / (ms / 1e3) / 1e9, 4), "unit": UNIT,
            "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 3 ** r,
            "steps": steps, "ms_per_step": round(ms / steps, 3),
            "path": (f"compact layout (gasket cells only, rho {rho}) written by the kernel "
                     f"straight into pinned host memory over the host link; bytes per step "
                     f"= the 3^{r} cells, one contiguous run")}


def measure_e2e(sg, torch, dev, stream, w, grp, steps):
    """The same metric through the public API with the grid in pinned host
    memory: every step copies the grid in, runs the pass and copies it out."""
    r, n = w["r"], 1 << w["r"]
    host = torch.zeros(n * n, dtype=torch.uint8, pin_memory=True)
    dgrid = torch.empty(n * n, dtype=torch.uint8, device=dev)

    def step():
        sg.map_write_host(host, dgrid, r, w["rho"], w["map"], w["value"], w["seed"], stream,
                          order=w["order"], store=w["store"])

    step()
    torch.cuda.synchronize(dev)
    grp.barrier()
    ms, _ = time_launches(step, steps, stream)
    ms = grp.max(ms)
    nbytes = n * n
    del host, dgrid
    return {"value": round(grp.world * 3 ** r * steps / (ms / 1e3) / 1e9, 4), "unit": UNIT,
            "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
            "steps": steps, "ms_per_step": round(ms / steps, 3),
            "path": "grid copied from pinned host memory to the device, written, copied back"}


def cpu_baseline(w):
    """The CPU oracle, as it stands, on the whole level-16 uint8 grid: one
    single-threaded brute-force pass (about 10 s)."""
    import numpy as np
    import oracle
    r, n = w["r"], 1 << w["r"]
    grid = np.zeros((n, n), dtype=np.uint8)
    t0 = time.perf_counter()
    oracle.map_write(r, grid, oracle.VAL_HASH, w["seed"])
    dt = time.perf_counter() - t0
    return {"value": round(3 ** r / dt / 1e9, 6), "unit": UNIT, "cores": 1,
            "kind": "oracle", "seconds": round(dt, 3),
            "sample": f"whole level-{r} uint8 grid ({n}x{n}), one pass, hash seed {w['seed']}",
            "host": _host_desc()}


def _oracle_band(job):
    """One row band of the oracle's write pass (a worker of the all-cores
    baseline): rows [y0, y1) of the level-r grid into a band buffer."""
    import numpy as np
    import oracle
    r, y0, y1, seed = job
    buf = np.zeros((y1 - y0, 1 << r), dtype=np.uint8)
    oracle.map_write(r, buf, oracle.VAL_HASH, seed, y0=y0, y1=y1)
    return y1 - y0


def cpu_baseline_all_cores(w, band=1024):
    """The same oracle pass over the whole level-16 grid, its row bands spread
    over one process per host core (a spawn-context pool: this process has
    used the GPU already, and a forked worker could hang).  The oracle's code
    is unchanged; only its bands run side by side."""
    import multiprocessing as mp
    r, n = w["r"], 1 << w["r"]
    cores = os.cpu_count() or 1
    jobs = [(r, y0, y0 + band, w["seed"]) for y0 in range(0, n, band)]
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_band, [(r, 0, 1, w["seed"])] * cores)   # workers load the oracle
        t0 = time.perf_counter()
        rows = sum(pool.map(_oracle_band, jobs, chunksize=1))
        dt = time.perf_counter() - t0
    assert rows == n
    return {"value": round(3 ** r / dt / 1e9, 6), "unit": UNIT, "cores": cores,
            "kind": "oracle", "seconds": round(dt, 3),
            "sample": (f"whole level-{r} uint8 grid ({n}x{n}), one pass, hash seed "
                       f"{w['seed']}, {n // band} bands of {band} rows over {cores} processes"),
            "host": _host_desc()}


def _host_desc():
    try:
        import platform
        return f"{platform.machine()}, {os.cpu_count()} cores"
    except Exception:
        return None


# --------------------------------------------------------------------------
# reference arm: the CPU oracle
# --------------------------------------------------------------------------
def band_cells(r: int, y0: int, y1: int) -> int:
    # row y of the level-r gasket holds the 2^(r - popcount(y)) subsets of ~y
    return sum(1 << (r - bin(y).count("1")) for y in range(y0, y1))


def run_reference(args, grp: Group):
    """The reference arm: the CPU oracle, as it stands, on the host's cores.
    A step is one band of 1024 rows of the level-16 uint8 grid per core, the
    bands run side by side in spawned processes (the oracle's code is not
    changed; only its row bands are spread over the cores)."""
    import multiprocessing as mp
    from paper_1706_04552_gb300 import workloads
    w = workloads.WRITE_HEADLINE
    r, n = w["r"], 1 << w["r"]
    band = 1024
    cores = os.cpu_count() or 1
    nb = n // band

    def jobs(i):
        first = (i * cores) % nb
        ys = [((first + c) % nb) * band for c in range(cores)]
        return [(r, y0, y0 + band, w["seed"]) for y0 in ys]

    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        pool.map(_oracle_band, [(r, 0, 1, w["seed"])] * cores)     # workers load the oracle
        for i in range(args.warmup):
            pool.map(_oracle_band, jobs(i), chunksize=1)
        t0 = time.perf_counter()
        cells = 0
        for i in range(args.steps):
            js = jobs(args.warmup + i)
            pool.map(_oracle_band, js, chunksize=1)
            cells += sum(band_cells(r, y0, y1) for _, y0, y1, _ in js)
        dt = time.perf_counter() - t0
    value = cells / dt / 1e9
    sample = (f"{args.steps} steps, each {cores} bands of {band} rows of the level-{r} uint8 "
              f"grid ({n} columns) in {cores} processes, hash seed {w['seed']}")
    return {
        "impl": "reference", "metric": METRIC, "value": round(value, 6), "unit": UNIT,
        "n_gpus": grp.world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": {"workload": (f"map-and-write, level {r} gasket in a {n}x{n} uint8 grid, "
                                f"hash(x,y) seed {w['seed']} (CPU oracle, row bands on "
                                f"{cores} cores)"),
                   "r": r, "n": n, "cells_per_step_mean": cells / args.steps},
        "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "cores": cores,
                         "kind": "oracle", "sample": sample, "host": _host_desc()},
        "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }


def main():
    args = parse_args()
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return 0
        grp = Group.__new__(Group)
        grp.world, grp.rank, grp.local, grp.dist, grp.backend = (
            int(os.environ.get("WORLD_SIZE", "1")), 0, 0, None, None)
        print(json.dumps(run_reference(args, grp)))
        return 0
    if args.paper_sweep:
        print(json.dumps(paper_sweep(args)))
        return 0
    if args.write_sweep:
        print(json.dumps(write_sweep(args)))
        return 0
    grp = Group()
    try:
        out = run_ours(args, grp)
        if grp.rank == 0:
            print(json.dumps(out))
    finally:
        grp.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
