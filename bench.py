"""Benchmark: Vietoris–Rips barcodes on one GB300 (or N replicas under torchrun).

Workload: 1000 points on a noisy 2-torus in R^3 (major radius 2, minor radius 1,
sigma 0.02), FP32 distance matrix, threshold 1.0, barcodes H0-H2 over Z/2.
A step is one full barcode computation (prologue, H0, and for d = 1, 2:
enumeration, apparent-pair test, sort, reduction, readout) on the distance
matrix already resident in HBM.  The unit is simplices: the number of
simplices of dimension 0..2 with diameter <= threshold.

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead (the
reference arm: a plain CPU implementation of the method, see oracle/).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "torus1000"
L2_FLUSH_BYTES = 256 << 20  # larger than the 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--profile", action="store_true",
                    help="warm-up calls then exactly one barcode call, for ncu launch lists and captures")
    return ap.parse_args()


def load_workload(name):
    from paper_1908_02518_gb300 import workloads as W
    return W.WORKLOADS[name]()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def cpu_baseline(w, budget_s=12.0):
    """The oracle as it stands, single-threaded on the host, repeated on the
    full workload until about budget_s seconds of CPU work."""
    import oracle
    oracle.build()
    d = w.dist
    t0 = time.perf_counter()
    runs = 0
    units = 0
    while True:
        r = oracle.barcodes(d, w.dim_max, w.threshold, w.p, method="coh")
        runs += 1
        units += sum(s["simplices"] for s in r.stats)
        if time.perf_counter() - t0 >= budget_s or runs >= 1000:
            break
    el = time.perf_counter() - t0
    return {"value": units / el, "unit": "simplices/s", "cores": 1, "kind": "oracle",
            "sample": f"{runs} full runs of the {w.name} workload (cohomology oracle, {el:.1f} s)"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = load_workload(args.workload)
    import oracle
    oracle.build()
    units = None
    for _ in range(args.warmup):
        oracle.barcodes(w.dist, w.dim_max, w.threshold, w.p)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.barcodes(w.dist, w.dim_max, w.threshold, w.p)
        times.append(time.perf_counter() - t0)
        units = sum(s["simplices"] for s in r.stats)
    tot = sum(times)
    val = units * len(times) / tot
    line = {"impl": "reference", "metric": "rips_barcode_simplices_per_s", "value": val, "unit": "simplices/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": w.name, "n": w.n, "dim_max": w.dim_max,
                                             "threshold": w.threshold, "p": w.p, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": val, "unit": "simplices/s", "cores": 1, "kind": "oracle",
                             "sample": f"the full {w.name} workload per step"},
            "e2e": {"value": val, "unit": "simplices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    world, rank, local = dist_env()
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_1908_02518_gb300 as rg
    from paper_1908_02518_gb300 import _lib
    lib = _lib.load()

    w = load_workload(args.workload)
    n = w.n
    dev_d = torch.from_numpy(w.dist).cuda()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    if args.profile:
        for _ in range(args.warmup):
            rg.barcodes(dev_d, w.dim_max, w.threshold, w.p)
        torch.cuda.synchronize()
        res = rg.barcodes(dev_d, w.dim_max, w.threshold, w.p)
        torch.cuda.synchronize()
        print(json.dumps({"profile": w.name, "bars": len(res.bars), "phase_ms": res.phase_ms}))
        return 0

    # warm-up (also sizes the workspace)
    for _ in range(max(3, args.warmup)):
        res = rg.barcodes(dev_d, w.dim_max, w.threshold, w.p)
    units_per_dim = [s["simplices"] for s in res.stats[0]]
    units = sum(units_per_dim)

    # timed region: K steps, each bracketed by events on the launching stream,
    # with an L2 flush (not timed) between steps
    clocks = Clocks(local) if rank == 0 else None
    rg.launch_count(reset=True)
    barrier()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    phase = []
    for k in range(args.steps):
        flush.zero_()
        ev[k][0].record(stream)
        res = rg.barcodes(dev_d, w.dim_max, w.threshold, w.p)
        ev[k][1].record(stream)
        phase.append(res.phase_ms)
    barrier()
    launches = rg.launch_count()
    ck = clocks.stop() if clocks else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = world * units * args.steps / (total_ms / 1000.0)
    per_dim = []
    for d in range(w.dim_max + 1):
        ph = statistics.median(p[d] for p in phase)
        per_dim.append({"dim": d, "simplices": units_per_dim[d], "phase_ms": ph,
                        "simplices_per_s": units_per_dim[d] / (ph / 1000.0) if ph > 0 else None})

    # dominant kernel class, timed live with events on the call's stream
    rg.set_kernel_timing(True)
    km = {}
    kr = 3
    for _ in range(kr):
        flush.zero_()
        r = rg.barcodes(dev_d, w.dim_max, w.threshold, w.p)
        for name, (ms, regions) in r.kernel_ms.items():
            a = km.setdefault(name, [0.0, 0])
            a[0] += ms / kr
            a[1] += regions / kr
    rg.set_kernel_timing(False)
    dom = max(km, key=lambda x: km[x][0])
    stats = res.stats[0]
    # algorithmic bytes of the dominant kernel class per timed region
    algo_bytes = None
    if dom == "apparent":
        tested = sum(s["simplices"] for s in stats[1:])
        cols = sum(s["columns"] for s in stats[1:])
        algo_bytes = (12 * tested + 8 * cols) / max(km[dom][1], 1)
    elif dom == "reduce":
        cols = sum(s["columns"] for s in stats[1:])
        algo_bytes = 24 * cols / max(km[dom][1], 1)
    elif dom == "prologue":
        algo_bytes = (4 * n * n + 4 * n * n) / max(km[dom][1], 1)
    elif dom == "enumerate":
        algo_bytes = sum(12 * s["simplices"] for s in stats[2:]) / max(km[dom][1], 1)
    peak, peak_kind = peaks()
    roof = None
    if algo_bytes is not None and km[dom][0] > 0:
        per_region_ms = km[dom][0] / max(km[dom][1], 1)
        achieved = algo_bytes / (per_region_ms / 1000.0) / 1e9
        roof = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                "region_ms": per_region_ms, "algorithmic_bytes": algo_bytes}

    # end to end through the C ABI with host buffers (copies inside the timed region)
    pinned = torch.from_numpy(w.dist).pin_memory()
    host = pinned.numpy()
    e2e_t = []
    nbars = 0
    for k in range(max(3, args.steps // 2) + 2):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = rg.barcodes(host, w.dim_max, w.threshold, w.p)
        t1 = time.perf_counter()
        if k >= 2:
            e2e_t.append(t1 - t0)
        nbars = len(r.bars)
    e2e_s = sum(e2e_t) / len(e2e_t)
    e2e = {"value": world * units / e2e_s, "unit": "simplices/s", "h2d_bytes_per_step": 4 * n * n,
           "d2h_bytes_per_step": 32 * nbars, "ms_per_step": 1000 * e2e_s}

    if rank == 0:
        cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline(w)
        line = {"metric": "rips_barcode_simplices_per_s", "value": value, "unit": "simplices/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64 integer ranks and indices; f32 values",
                "data": "synthetic",
                "config": {"workload": w.name, "n": n, "dim_max": w.dim_max, "threshold": w.threshold, "p": w.p,
                           "parallelism": f"replicas{world}" if world > 1 else "single",
                           "l2": "flushed between steps (256 MiB write)"},
                "per_dim": per_dim, "barcode_ms": ms_per_step, "bars": nbars,
                "kernel_ms": {k: v[0] for k, v in km.items()},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": ck}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
