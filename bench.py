#!/usr/bin/env python3
"""Benchmark: D8 directions + unit up-slope counts on a 32768 x 32768 pit-free
fractal DEM (1.07 G cells), one pipeline call per step (direction stencil,
tile pass, combine, finalise).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload NAME] [--tile T] [--no-cpu-baseline] [--no-extras]

Prints ONE JSON line (rank 0).  `value` is cells/s with the DEM resident in
HBM (device-timed with CUDA events, max over ranks); `e2e` is the same metric
through the public API with pinned host buffers, host->device copy of z and
device->host copy of the directions and counts inside the timed region;
`roofline` is the dominant kernel's algorithmic bytes per launch over its
event-timed duration against the measured HBM copy bandwidth; `cpu_baseline`
times the CPU oracle on a bounded crop of the same DEM.  On one GPU the line
also carries `batched` (512 DEMs of uneven sizes in one graph-captured
persistent pipeline, autotuned tile, beside the same DEMs one call at a time)
and `fwd_bwd` (weighted forward + backward at 8192 x 8192 beside the plain
pipeline on the same DEM).  With torchrun (N>1) every rank processes its own
replica of the workload (independent DEMs, no collective on the data path):
weak scaling.
"""
from __future__ import annotations

import argparse
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
KERNEL_SOURCE = {"flowdir": "d8_flowdir.cu", "tile_up": "d8_unit.cu", "tile_down": "d8_unit.cu"}


def measured_traffic(stage: str):
    """DRAM bytes per cell of a stage's kernel from the committed ncu summary,
    or None when that kernel's source changed since the capture."""
    import hashlib

    prof = os.path.join(ROOT, "profiles", "tile_kernels_fractal_8192.md")
    src = os.path.join(ROOT, "paper_1605_05773_gb300", "csrc", KERNEL_SOURCE.get(stage, ""))
    try:
        text = open(prof).read().split()
        sha = hashlib.sha1(open(src, "rb").read()).hexdigest()[:12]
    except OSError:
        return None
    ok = any(text[k] == "kernel_source_sha1" and text[k + 1] == KERNEL_SOURCE[stage] and text[k + 2] == sha
             for k in range(len(text) - 2))
    if not ok:
        return None
    for k in range(len(text) - 2):
        if text[k] == "scaled_traffic_bytes_per_cell" and text[k + 1] == stage:
            return float(text[k + 2])
    return None


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


def oracle_sample(z, side: int):
    """Time the CPU oracle (directions + queue method) on a side x side crop."""
    import numpy as np

    import oracle

    crop = np.ascontiguousarray(z[:side, :side])
    t0 = time.perf_counter()
    d = oracle.flowdir(crop)
    oracle.accumulate(d)
    return time.perf_counter() - t0, crop.size


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


def run_batched(dev, stream, steps: int):
    """The 512-DEM batch (sides log-uniform in [128, 4096], aspect up to 1:4)
    through the graph-captured persistent pipeline with the autotuned tile,
    beside the same DEMs run one call at a time."""
    from concurrent.futures import ThreadPoolExecutor

    import torch

    import demgen
    import paper_1605_05773_gb300 as lib
    from tests.gpu_util import recursion_residual_gpu, terminal_sum_gpu

    shapes = demgen.batch_shapes(512)
    with ThreadPoolExecutor(max(1, min(16, os.cpu_count() or 1))) as ex:  # the C generator releases the GIL
        zs = list(ex.map(lambda a: demgen.fractal(a[1][0], a[1][1], seed=2000 + a[0]), enumerate(shapes)))
    cells = sum(h * w for h, w in shapes)
    zt = [torch.from_numpy(z).to(dev) for z in zs]
    del zs
    dirs = [torch.empty(s, dtype=torch.uint8, device=dev) for s in shapes]
    As = [torch.empty(s, dtype=torch.uint32, device=dev) for s in shapes]
    tile, tune_ms = lib.autotune_batch(zt, dirs, As)
    plan = lib.BatchPlan(shapes, dev)
    for _ in range(2):
        plan.run(zt, dirs, As)
    torch.cuda.synchronize(dev)
    if lib.get_status(dev) != "OK":
        raise RuntimeError("batched run: device status")
    ms = _event_ms(lambda: plan.run(zt, dirs, As), steps, stream)
    ok = all(recursion_residual_gpu(dirs[k], As[k]) == 0 and terminal_sum_gpu(dirs[k], As[k]) == h * w
             for k, (h, w) in enumerate(shapes) if k % 32 == 0)

    def one_by_one():
        for k in range(len(shapes)):
            lib.flowdir_accumulate(zt[k], "steepest", dir=dirs[k], A=As[k])

    one_by_one()
    ms_single = _event_ms(one_by_one, 2, stream)
    plan.close()
    return {"workload": "batch_512", "description": "512 pit-free fractal DEMs, sides log-uniform in [128, 4096], "
                                                    "aspect 1:1-1:4, one graph-captured persistent pipeline",
            "dems": len(shapes), "cells": cells, "tile": tile, "autotune_ms": tune_ms, "steps": steps,
            "value": cells / (ms / 1e3), "unit": "cells/s", "ms_per_step": ms,
            "unbatched": {"value": cells / (ms_single / 1e3), "ms_per_step": ms_single,
                          "how": "the same 512 DEMs through d8_flowdir_accumulate, one call per DEM, same tile"},
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


def run_ours(args, world, rank, local):
    import numpy as np
    import torch

    import demgen
    import paper_1605_05773_gb300 as lib

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    H, W, desc = WORKLOADS[args.workload]
    cells = H * W
    z_host = demgen.fractal(H, W)  # replicas: every rank gets the same recipe
    lib.set_tile(args.tile)
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

    # dominant kernel's roofline (algorithmic bytes / event-timed duration)
    peak, peak_kind = measured_peaks()
    dom = max((s for s in stages if stages[s][1] > 0 and s in ALG_BYTES), key=lambda s: stages[s][0])
    dom_ms = stages[dom][0] / args.steps
    achieved = ALG_BYTES[dom] * cells / (dom_ms / 1e3) / 1e9
    tb = measured_traffic(dom)
    launches = sum(v[1] for v in stages.values())

    # end to end through the public API: pinned host z in, dirs + counts out
    e2e_steps = max(1, min(args.steps, 5))
    zh = torch.from_numpy(z_host).pin_memory()
    dh = torch.empty((H, W), dtype=torch.uint8).pin_memory()
    Ah = torch.empty((H, W), dtype=torch.int32).pin_memory()
    torch.cuda.synchronize(dev)
    barrier(world)
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(e2e_steps):
        z.copy_(zh, non_blocking=True)
        lib.flowdir_accumulate(z, "steepest", dir=d, A=A)
        dh.copy_(d, non_blocking=True)
        Ah.copy_(A.view(torch.int32), non_blocking=True)
    f1.record(stream)
    torch.cuda.synchronize(dev)
    e2e_ms = max_over_ranks(f0.elapsed_time(f1), world, dev)
    e2e_val = world * cells * e2e_steps / (e2e_ms / 1e3)

    if rank == 0:
        # correctness guard on the timed buffers: Eq. 1 recursion and conservation
        from tests.gpu_util import recursion_residual_gpu, terminal_sum_gpu

        ok = recursion_residual_gpu(d, A) == 0 and terminal_sum_gpu(d, A) == cells
        del z
        cpu = None
        if not args.no_cpu_baseline:
            side = min(H, W, 8192)
            t, n = oracle_sample(z_host, side)
            cpu = {"value": n / t, "unit": "cells/s", "cores": 1, "kind": "oracle",
                   "sample": f"{side}x{side} crop of the workload DEM (oracle directions + one-worker queue method)"}
        line = {
            "metric": "cells_per_second", "value": value, "unit": "cells/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32 dirs, u32 counts", "data": "synthetic",
            "config": {"workload": args.workload, "description": desc, "H": H, "W": W, "tile": args.tile,
                       "l2": "inputs larger than L2 (4.3 GB z per step, 129 MB L2)", "parity_guard": ok},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": (tb * cells if tb else None),
                         "traffic_note": "ncu dram bytes per cell at 8192^2 (profiles/tile_kernels_fractal_8192.md) x cells; "
                                         "null when the kernel changed since that capture",
                         "peak_kind": peak_kind,
                         "alg_bytes_per_cell": ALG_BYTES[dom], "ms_per_launch": dom_ms},
            "pipeline_roofline": {"alg_bytes_per_cell": PIPE_BYTES,
                                  "achieved": PIPE_BYTES * cells / (ms_max / args.steps / 1e3) / 1e9,
                                  "frac": PIPE_BYTES * cells / (ms_max / args.steps / 1e3) / 1e9 / peak},
            "stages_ms_per_step": {k: v[0] / args.steps for k, v in stages.items() if v[1]},
            "gpu_launches": launches,
            "e2e": {"value": e2e_val, "unit": "cells/s", "h2d_bytes_per_step": 4 * cells,
                    "d2h_bytes_per_step": 5 * cells, "steps": e2e_steps},
            "cpu_baseline": cpu,
            "clocks": clk,
        }
        if world == 1 and not args.no_extras:
            lib.set_profiling(False, dev)
            line["batched"] = run_batched(dev, stream, max(3, min(args.steps, 5)))
            lib.set_tile(args.tile)
            line["fwd_bwd"] = run_fwd_bwd(dev, stream, max(3, min(args.steps, 10)))
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
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched and fwd+bwd lines")
    args = ap.parse_args()
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
