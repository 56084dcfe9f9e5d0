#!/usr/bin/env python3
"""Benchmark: D8 directions + unit up-slope counts on a 32768 x 32768 pit-free
fractal DEM (1.07 G cells), one pipeline call per step (direction stencil,
tile pass, combine, finalise).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--tile T] [--strategy S] [--no-cpu-baseline]
                  [--no-extras]

Prints ONE JSON line (rank 0).  `value` is cells/s with the DEM resident in
HBM (device-timed with CUDA events, max over ranks).  `e2e` is the same metric
through the public API with pinned host buffers: every step copies its DEM
in, runs the call and copies the directions and counts out; steps are
pipelined (the next DEM's copy in and the previous results' copy out overlap
the current call, on their own streams), and `e2e.serial` gives the same with
nothing overlapped.  `roofline` is the dominant kernel's algorithmic bytes per
launch over its event-timed duration against the measured HBM copy
bandwidth; `cpu_baseline` times the CPU oracle (one core) and
`cpu_reference_mt` the multi-core CPU reference (every core this process may
use) on a bounded crop of the same DEM.  On one GPU the line also carries
`batched` (512 DEMs of uneven sizes in one graph-captured persistent
pipeline, tile and strategy autotuned, beside the same DEMs one call at a
time), `fwd_bwd` (weighted forward + backward at 8192 x 8192 beside the plain
pipeline on the same DEM) and `workloads` (the other configurations: the
8192^2 tilted plane, the 8192^2 serpentine as a DEM and as a direction field,
and the 16384 x 65536 fractal, each with the combine's link-graph statistics
under the queue walk and under pointer jumping), and `fill` (pit and flat
removal on the raw 8192^2 and 32768^2 fractals).  With torchrun (N>1) every
rank processes its own replica of the workload (independent DEMs, no
collective on the data path): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (H, W, description)
    "fractal_32768": (32768, 32768, "32768x32768 fp32 pit-free fractal DEM (diamond-square H=0.8, 0-1000 m, "
                                    "Priority-Flood+eps 1e-3 m), steepest rule, unit weights, uint8 dirs + "
                                    "uint32 counts"),
    "fractal_8192": (8192, 8192, "8192x8192 fp32 pit-free fractal DEM, steepest rule, unit weights"),
    "fractal_512": (512, 512, "512x512 fp32 pit-free fractal DEM, steepest rule, unit weights"),
}
# Algorithmic bytes per cell of the stages whose traffic does not depend on
# the data: the direction stencil reads z (4) and writes dir (1); the tile
# pass reads dir (1) and writes the in-tile counts (4).  The finalising pass
# reads dir (1) and rewrites A only where inflow from other tiles arrives.
ALG_BYTES = {"flowdir": 5.0, "tile_up": 5.0}
PIPE_BYTES = 9.0  # z in (4) + dir out (1) + A out (4) per cell for the whole path
TRAFFIC_FILE = os.path.join("profiles", "ncu_traffic.json")


def measured_traffic(stage: str):
    """DRAM bytes per cell of a stage's kernel from the committed ncu figures
    (profiles/ncu_traffic.json), or None when that kernel's source changed
    since the capture."""
    try:
        with open(os.path.join(ROOT, TRAFFIC_FILE)) as f:
            j = json.load(f)
        src = j["kernel_source"][stage]
        with open(os.path.join(ROOT, "paper_1605_05773_gb300", "csrc", src), "rb") as f:
            sha = hashlib.sha1(f.read()).hexdigest()[:12]
    except (OSError, ValueError, KeyError):
        return None
    if j.get("kernel_source_sha1", {}).get(src) != sha:
        return None
    v = j.get("dram_bytes_per_cell", {}).get(stage)
    return float(v) if v is not None else None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = [r for r in self.rows if len(r) >= 9]
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, n in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return world, rank, local


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


# ---- result guards on the timed buffers (plain torch, independent of libd8)
_DI = (-1, -1, 0, 1, 1, 1, 0, -1)
_DJ = (0, 1, 1, 1, 0, -1, -1, -1)


def recursion_residual(dir, A) -> int:
    """max |A(p) - 1 - sum of A over the cells draining into p| (Eq. 1) in int64."""
    import torch

    with torch.no_grad():
        H, W = dir.shape
        dpad = torch.full((H + 2, W + 2), 255, dtype=torch.uint8, device=dir.device)
        dpad[1:-1, 1:-1] = dir
        Apad = torch.zeros((H + 2, W + 2), dtype=torch.int64, device=dir.device)
        Apad[1:-1, 1:-1] = A.view(torch.int32).to(torch.int64) & 0xFFFFFFFF
        inflow = torch.zeros((H, W), dtype=torch.int64, device=dir.device)
        for k in range(8):
            nd = dpad[1 + _DI[k]:1 + _DI[k] + H, 1 + _DJ[k]:1 + _DJ[k] + W]
            na = Apad[1 + _DI[k]:1 + _DI[k] + H, 1 + _DJ[k]:1 + _DJ[k] + W]
            inflow += torch.where(nd == ((k + 4) % 8), na, 0)
            del nd, na
        return int((Apad[1:-1, 1:-1] - 1 - inflow).abs().max().item())


def terminal_sum(dir, A) -> int:
    """Sum of A over the cells where a path ends (codes 8/9, or a target off the grid)."""
    import torch

    with torch.no_grad():
        H, W = dir.shape
        i = torch.arange(H, device=dir.device).view(H, 1)
        j = torch.arange(W, device=dir.device).view(1, W)
        term = dir >= 8
        for k in range(8):
            off = ((i + _DI[k] < 0) | (i + _DI[k] >= H)) | ((j + _DJ[k] < 0) | (j + _DJ[k] >= W))
            term |= (dir == k) & off
        return int((A.view(torch.int32).to(torch.int64) & 0xFFFFFFFF)[term].sum().item())


def guard(dir, A) -> bool:
    H, W = dir.shape
    return recursion_residual(dir, A) == 0 and terminal_sum(dir, A) == H * W


# ---- CPU baselines
def oracle_sample(z, side: int):
    """Time the CPU oracle (directions + queue method, one core) on a side x side crop."""
    import numpy as np

    import oracle

    crop = np.ascontiguousarray(z[:side, :side])
    t0 = time.perf_counter()
    d = oracle.flowdir(crop)
    oracle.accumulate(d)
    return time.perf_counter() - t0, crop.size


def cpuref_sample(z, side: int):
    """Time the multi-core CPU reference on a side x side crop (median of 3)."""
    import numpy as np

    import cpuref

    crop = np.ascontiguousarray(z[:side, :side])
    ts = []
    for _ in range(3):
        t0 = time.perf_counter()
        d = cpuref.flowdir(crop)
        cpuref.accumulate(d)
        ts.append(time.perf_counter() - t0)
    return sorted(ts)[1], crop.size, cpuref.cores()


def run_reference(args, world, rank):
    """The CPU oracle on the host cores: the reference arm of this benchmark."""
    H, W, desc = WORKLOADS[args.workload]
    if rank != 0:
        return 0
    import demgen

    z = demgen.fractal(H, W)
    side = min(H, W, 4096 if args.steps + args.warmup <= 12 else 2048)
    for _ in range(args.warmup):
        oracle_sample(z, side)
    tot, cells = 0.0, 0
    for _ in range(args.steps):
        t, n = oracle_sample(z, side)
        tot += t
        cells += n
    v = cells / tot
    line = {
        "impl": "reference", "metric": "cells_per_second", "value": v, "unit": "cells/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 dirs, u64 counts",
        "data": "synthetic",
        "config": {"workload": args.workload, "description": desc, "H": H, "W": W},
        "cpu_baseline": {"value": v, "unit": "cells/s", "cores": 1, "kind": "oracle",
                         "sample": f"{side}x{side} crop of the workload DEM per step (oracle directions + "
                                   f"one-worker queue method)"},
        "e2e": {"value": v, "unit": "cells/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _event_ms(fn, reps, stream):
    import torch

    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def run_e2e(lib, z_host, H, W, steps, dev, world):
    """Directions and counts end to end through the public call, K steps, each
    step copying its DEM in from pinned host memory and its directions and
    counts out to pinned host memory.  Pipelined: copies in on one stream,
    the call on the compute stream, copies out on a third, two device buffer
    sets alternating, so step k+1's copy in and step k-1's copy out overlap
    step k's call.  Also timed with everything on one stream (serial)."""
    import torch

    cells = H * W
    zh = torch.from_numpy(z_host).pin_memory()
    dh = [torch.empty((H, W), dtype=torch.uint8).pin_memory() for _ in range(2)]
    Ah = [torch.empty((H, W), dtype=torch.int32).pin_memory() for _ in range(2)]
    zd = [torch.empty((H, W), dtype=torch.float32, device=dev) for _ in range(2)]
    dd = [torch.empty((H, W), dtype=torch.uint8, device=dev) for _ in range(2)]
    Ad = [torch.empty((H, W), dtype=torch.uint32, device=dev) for _ in range(2)]
    s_in, s_cmp, s_out = (torch.cuda.Stream(dev) for _ in range(3))
    torch.cuda.synchronize(dev)

    def pipelined(k_steps):
        copied = [torch.cuda.Event() for _ in range(k_steps)]
        computed = [torch.cuda.Event() for _ in range(k_steps)]
        drained = [torch.cuda.Event() for _ in range(k_steps)]
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s_in)
        s_cmp.wait_event(e0)
        s_out.wait_event(e0)
        for k in range(k_steps):
            b = k & 1
            with torch.cuda.stream(s_in):
                if k >= 2:
                    s_in.wait_event(computed[k - 2])  # the call of step k-2 is done with zd[b]
                zd[b].copy_(zh, non_blocking=True)
                copied[k].record(s_in)
            with torch.cuda.stream(s_cmp):
                s_cmp.wait_event(copied[k])
                if k >= 2:
                    s_cmp.wait_event(drained[k - 2])  # dd[b], Ad[b] copied out
                lib.flowdir_accumulate(zd[b], "steepest", dir=dd[b], A=Ad[b])
                computed[k].record(s_cmp)
            with torch.cuda.stream(s_out):
                s_out.wait_event(computed[k])
                dh[b].copy_(dd[b], non_blocking=True)
                Ah[b].copy_(Ad[b].view(torch.int32), non_blocking=True)
                drained[k].record(s_out)
        s_in.wait_event(drained[k_steps - 1])
        e1.record(s_in)
        e1.synchronize()
        return e0.elapsed_time(e1)

    def serial(k_steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s_cmp):
            e0.record(s_cmp)
            for _ in range(k_steps):
                zd[0].copy_(zh, non_blocking=True)
                lib.flowdir_accumulate(zd[0], "steepest", dir=dd[0], A=Ad[0])
                dh[0].copy_(dd[0], non_blocking=True)
                Ah[0].copy_(Ad[0].view(torch.int32), non_blocking=True)
            e1.record(s_cmp)
        e1.synchronize()
        return e0.elapsed_time(e1)

    pipelined(2)  # warm-up
    barrier(world)
    ms_p = max_over_ranks(pipelined(steps), world, dev)
    barrier(world)
    ms_s = max_over_ranks(serial(steps), world, dev)
    ok = guard(dd[(steps - 1) & 1], Ad[(steps - 1) & 1])
    for t in (zd, dd, Ad):
        t.clear()
    return {"value": world * cells * steps / (ms_p / 1e3), "unit": "cells/s", "h2d_bytes_per_step": 4 * cells,
            "d2h_bytes_per_step": 5 * cells, "steps": steps, "ms_per_step": ms_p / steps,
            "how": "public call with pinned host buffers; copies in, the call and copies out on three streams, "
                   "two device buffer sets, consecutive steps overlapped",
            "parity_guard": ok,
            "serial": {"value": world * cells * steps / (ms_s / 1e3), "ms_per_step": ms_s / steps,
                       "how": "the same with copy in, call and copy out back to back on one stream"}}


def run_batched(dev, stream, steps: int):
    """The 512-DEM batch (sides log-uniform in [128, 4096], aspect up to 1:4)
    through the graph-captured persistent pipeline with the autotuned tile and
    strategy, beside the same DEMs run one call at a time."""
    from concurrent.futures import ThreadPoolExecutor

    import torch

    import demgen
    import paper_1605_05773_gb300 as lib

    shapes = demgen.batch_shapes(512)
    with ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:  # the C generator releases the GIL
        zs = list(ex.map(lambda a: demgen.fractal(a[1][0], a[1][1], seed=2000 + a[0]), enumerate(shapes)))
    cells = sum(h * w for h, w in shapes)
    zt = [torch.from_numpy(z).to(dev) for z in zs]
    del zs
    dirs = [torch.empty(s, dtype=torch.uint8, device=dev) for s in shapes]
    As = [torch.empty(s, dtype=torch.uint32, device=dev) for s in shapes]
    tile, strat, tune = lib.autotune_batch(zt, dirs, As)
    table = {str(t): {s: tune[(t, s)] for s in lib.STRATEGIES} for t in (32, 64, 128)}
    plan = lib.BatchPlan(shapes, dev)
    for _ in range(2):
        plan.run(zt, dirs, As)
    torch.cuda.synchronize(dev)
    if lib.get_status(dev) != "OK":
        raise RuntimeError("batched run: device status")
    ms = _event_ms(lambda: plan.run(zt, dirs, As), steps, stream)
    ok = all(guard(dirs[k], As[k]) for k in range(0, len(shapes), 32))

    def one_by_one():
        for k in range(len(shapes)):
            lib.flowdir_accumulate(zt[k], "steepest", dir=dirs[k], A=As[k])

    one_by_one()
    ms_single = _event_ms(one_by_one, 2, stream)
    plan.close()
    return {"workload": "batch_512", "description": "512 pit-free fractal DEMs, sides log-uniform in [128, 4096], "
                                                    "aspect 1:1-1:4, one graph-captured persistent pipeline",
            "dems": len(shapes), "cells": cells, "tile": tile, "strategy": strat,
            "autotune_ms": table, "autotune_how": "median of 5 graph replays per (tile, strategy) point",
            "steps": steps, "value": cells / (ms / 1e3), "unit": "cells/s", "ms_per_step": ms,
            "unbatched": {"value": cells / (ms_single / 1e3), "ms_per_step": ms_single,
                          "how": "the same 512 DEMs through d8_flowdir_accumulate, one call per DEM, same tile "
                                 "and strategy"},
            "parity_guard": ok}


def run_fwd_bwd(dev, stream, steps: int):
    """Weighted forward + hand-written backward on the 8192 x 8192 fractal with
    lognormal weights and normal cotangents, beside the plain unit pipeline on
    the same DEM."""
    import torch

    import demgen
    import paper_1605_05773_gb300 as lib

    n = 8192
    z = torch.from_numpy(demgen.fractal(n, n)).to(dev)
    d = lib.flowdir(z)
    w = torch.from_numpy(demgen.lognormal_weights(n, n, 11)).to(dev)
    c = torch.from_numpy(demgen.normal_cotangent(n, n, 12)).to(dev)
    A = torch.empty((n, n), dtype=torch.float32, device=dev)
    dw = torch.empty((n, n), dtype=torch.float32, device=dev)
    Au = torch.empty((n, n), dtype=torch.uint32, device=dev)
    fwd = lambda: lib.accumulate_weighted(d, w, out=A)  # noqa: E731
    bwd = lambda: lib.accumulate_backward(d, c, out=dw)  # noqa: E731
    plain = lambda: lib.flowdir_accumulate(z, "steepest", dir=d, A=Au)  # noqa: E731
    for _ in range(3):
        fwd()
        bwd()
        plain()
    torch.cuda.synchronize(dev)
    if lib.get_status(dev) != "OK":
        raise RuntimeError("fwd/bwd run: device status")
    ms_fwd = _event_ms(fwd, steps, stream)
    ms_bwd = _event_ms(bwd, steps, stream)
    ms_fb = _event_ms(lambda: (fwd(), bwd()), steps, stream)
    ms_plain = _event_ms(plain, steps, stream)
    cells = n * n
    return {"workload": "weighted_8192", "description": "8192x8192 pit-free fractal, fp32 lognormal(0,1) weights, "
                                                        "fp32 N(0,1) cotangents; weighted forward + backward",
            "cells": cells, "steps": steps, "value": cells / (ms_fb / 1e3), "unit": "cells/s",
            "ms_per_step": ms_fb, "fwd_ms": ms_fwd, "bwd_ms": ms_bwd,
            "plain": {"value": cells / (ms_plain / 1e3), "ms_per_step": ms_plain,
                      "how": "d8_flowdir_accumulate (unit counts, directions included) on the same DEM"}}


def run_fill(dev, steps: int):
    """Pit and flat removal (d8_fill) on the raw 8192^2 and 32768^2 fractals
    (the generator's diamond-square output before its own fill), beside the
    oracle's priority flood on one host core over a 2048^2 crop."""
    import numpy as np
    import torch

    import demgen
    import oracle
    import paper_1605_05773_gb300 as lib

    out = {}
    for n, reps in ((8192, max(2, steps)), (32768, 2)):
        z = demgen.fractal_raw(n, n, demgen.SEED_BASE)
        zt = torch.from_numpy(z).to(dev)
        F = torch.empty_like(zt)
        lib.fill(zt, 1e-3, out=F)
        torch.cuda.synchronize(dev)
        if lib.get_status(dev) != "OK":
            raise RuntimeError("fill: device status")
        t0 = time.perf_counter()
        for _ in range(reps):
            _, rounds = lib.fill(zt, 1e-3, out=F, return_rounds=True)
        torch.cuda.synchronize(dev)
        ms = (time.perf_counter() - t0) * 1e3 / reps
        raised = int((F != zt).sum().item())
        out[f"fractal_raw_{n}"] = {"ms_per_fill": ms, "value": n * n / (ms / 1e3), "unit": "cells/s",
                                   "tile_rounds": rounds, "cells_raised": raised,
                                   "timing": "host wall clock around the synchronous call (it checks convergence "
                                             "on the host every 16 rounds)"}
        del zt, F
    crop = np.ascontiguousarray(demgen.fractal_raw(2048, 2048, demgen.SEED_BASE))
    t0 = time.perf_counter()
    oracle.fill_eps(crop, 1e-3)
    out["cpu_oracle_2048"] = {"value": crop.size / (time.perf_counter() - t0), "unit": "cells/s", "cores": 1,
                              "kind": "oracle (priority flood with a binary heap)"}
    return out


def run_workloads(dev, stream, steps: int):
    """The other configurations, each timed under the queue walk (strategy
    "ring") and under top-level pointer jumping ("jump"), with the combine's
    link-graph statistics (group levels, top-level exits, and the rounds that
    bound the depth of the top-level link graph: how far the flow paths wind
    across the tiles)."""
    import torch

    import demgen
    import paper_1605_05773_gb300 as lib

    cases = [
        ("plane_8192", "8192x8192 tilted plane (0.05 m/cell S, 0.02 m/cell E, +-0.01 m noise) + eps-fill, "
                       "directions and counts", lambda: demgen.plane(8192, 8192), "z"),
        ("serpentine_dem_8192", "8192x8192 realisable serpentine DEM (width-1 channels on odd rows, one outlet), "
                                "directions and counts", lambda: demgen.serpentine_dem(8192, 8192), "z"),
        ("serpentine_dirs_8192", "8192x8192 boustrophedon direction field: one path through all 2^26 cells, "
                                 "counts only", lambda: demgen.serpentine_dirs(8192, 8192), "dir"),
        ("fractal_16384x65536", "16384x65536 pit-free fractal DEM (4x1 lattice of diamond-square squares), "
                                "directions and counts", lambda: demgen.fractal(16384, 65536), "z"),
    ]
    out = {}
    for name, desc, make, kind in cases:
        host = make()
        H, W = host.shape
        x = torch.from_numpy(host).to(dev)
        del host
        d = x if kind == "dir" else torch.empty((H, W), dtype=torch.uint8, device=dev)
        A = torch.empty((H, W), dtype=torch.uint32, device=dev)
        call = (lambda: lib.accumulate(d, out=A)) if kind == "dir" else \
            (lambda: lib.flowdir_accumulate(x, "steepest", dir=d, A=A))
        entry = {"description": desc, "H": H, "W": W, "cells": H * W}
        for strat in ("ring", "jump"):
            lib.set_strategy(strat, dev)
            call()
            torch.cuda.synchronize(dev)
            if lib.get_status(dev) != "OK":
                raise RuntimeError(f"{name}: device status")
            stats = lib.combine_stats(dev)
            reps = steps if W * H <= (1 << 28) else max(2, steps // 2)
            ms = _event_ms(call, reps, stream)
            entry[strat] = {"ms_per_step": ms, "value": H * W / (ms / 1e3), "unit": "cells/s", "combine": stats}
        entry["parity_guard"] = guard(d, A)
        lib.set_strategy("ring", dev)
        out[name] = entry
        del x, d, A
        torch.cuda.empty_cache()
    return out


def run_ours(args, world, rank, local):
    import torch

    import demgen
    import paper_1605_05773_gb300 as lib

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    H, W, desc = WORKLOADS[args.workload]
    cells = H * W
    z_host = demgen.fractal(H, W)  # replicas: every rank gets the same recipe
    lib.set_tile(args.tile)
    lib.set_strategy(args.strategy)
    z = torch.from_numpy(z_host).to(dev)
    d = torch.empty((H, W), dtype=torch.uint8, device=dev)
    A = torch.empty((H, W), dtype=torch.uint32, device=dev)
    stream = torch.cuda.current_stream(dev)

    for _ in range(args.warmup):
        lib.flowdir_accumulate(z, "steepest", dir=d, A=A)
    torch.cuda.synchronize(dev)
    st = lib.get_status(dev)
    if st != "OK":
        raise RuntimeError(f"device status {st}")
    lib.stage_times(dev)  # reset counters
    lib.set_profiling(True, dev)

    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        lib.flowdir_accumulate(z, "steepest", dir=d, A=A)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier(world)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    stages = lib.stage_times(dev)
    lib.set_profiling(False, dev)
    ms_max = max_over_ranks(ms, world, dev)
    value = world * cells * args.steps / (ms_max / 1e3)
    stats = lib.combine_stats(dev)
    ok = guard(d, A)

    # dominant kernel's roofline (algorithmic bytes / event-timed duration)
    peak, peak_kind = measured_peaks()
    dom = max((s for s in stages if stages[s][1] > 0 and s in ALG_BYTES), key=lambda s: stages[s][0])
    dom_ms = stages[dom][0] / args.steps
    achieved = ALG_BYTES[dom] * cells / (dom_ms / 1e3) / 1e9
    tb = measured_traffic(dom)
    launches = sum(v[1] for v in stages.values())

    del z
    torch.cuda.empty_cache()
    e2e = run_e2e(lib, z_host, H, W, max(6, min(args.steps, 12)), dev, world)  # fill and drain amortised

    if rank == 0:
        cpu = mt = None
        if not args.no_cpu_baseline:
            side = min(H, W, 8192)
            t, n = oracle_sample(z_host, side)
            cpu = {"value": n / t, "unit": "cells/s", "cores": 1, "kind": "oracle",
                   "sample": f"{side}x{side} crop of the workload DEM (oracle directions + one-worker queue method)"}
            t, n, nc = cpuref_sample(z_host, side)
            mt = {"value": n / t, "unit": "cells/s", "cores": nc,
                  "kind": "multi-core CPU reference (OpenMP direction pass + the paper's shared-memory queue method "
                          "with one queue per thread)",
                  "sample": f"{side}x{side} crop of the workload DEM, median of 3"}
        line = {
            "metric": "cells_per_second", "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 dirs, u32 counts", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "H": H, "W": W, "tile": args.tile,
                       "strategy": args.strategy,
                       "l2": "inputs larger than L2 (4.3 GB z per step, 129 MB L2)", "parity_guard": ok},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": (tb * cells if tb else None),
                         "traffic_note": f"ncu dram bytes per cell at 8192^2 ({TRAFFIC_FILE}) x cells; null when "
                                         "the kernel changed since that capture",
                         "peak_kind": peak_kind,
                         "alg_bytes_per_cell": ALG_BYTES[dom], "ms_per_launch": dom_ms},
            "pipeline_roofline": {"alg_bytes_per_cell": PIPE_BYTES,
                                  "achieved": PIPE_BYTES * cells / (ms_max / args.steps / 1e3) / 1e9,
                                  "frac": PIPE_BYTES * cells / (ms_max / args.steps / 1e3) / 1e9 / peak},
            "stages_ms_per_step": {k: v[0] / args.steps for k, v in stages.items() if v[1]},
            "combine": stats,
            "gpu_launches": launches,
            "e2e": e2e,
            "cpu_baseline": cpu,
            "cpu_reference_mt": mt,
            "clocks": clk,
        }
        extras = set() if args.no_extras else set(args.extras.split(",")) - {""}
        if world == 1 and extras:
            lib.set_profiling(False, dev)
            if "batched" in extras:
                line["batched"] = run_batched(dev, stream, max(3, min(args.steps, 5)))
                lib.set_tile(args.tile)
                lib.set_strategy(args.strategy)
            if "fwd_bwd" in extras:
                line["fwd_bwd"] = run_fwd_bwd(dev, stream, max(3, min(args.steps, 10)))
            if "workloads" in extras:
                line["workloads"] = run_workloads(dev, stream, max(3, min(args.steps, 10)))
            if "fill" in extras:
                line["fill"] = run_fill(dev, 3)
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="fractal_32768")
    ap.add_argument("--tile", type=int, default=64)
    ap.add_argument("--strategy", choices=["ring", "lane_mask", "jump"], default="ring")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--extras", default="batched,fwd_bwd,workloads,fill",
                    help="comma-separated extra lines to add (batched, fwd_bwd, workloads, fill)")
    ap.add_argument("--no-extras", action="store_true", help="add none of the extra lines")
    args = ap.parse_args()
    bad = set(args.extras.split(",")) - {"", "batched", "fwd_bwd", "workloads", "fill"}
    if bad:
        ap.error(f"unknown extras: {sorted(bad)}")
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        rc = run_reference(args, world, rank)
    else:
        rc = run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
