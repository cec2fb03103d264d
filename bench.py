"""Benchmark: Vietoris–Rips barcodes on one GB300 (or N replicas under torchrun).

Workload (default, the largest single-GPU configuration): 4096 Haar-random
rotations of R^3 flattened to points of R^9, FP32 distance matrix, threshold
1.4, barcodes H0-H2 over Z/2.  A step is one full barcode computation
(prologue, H0, and for d = 1, 2: enumeration, apparent-pair test, sort,
reduction, readout) on the distance matrix already resident in HBM.  The unit
is simplices: the number of simplices of dimension 0..2 with diameter <=
threshold.  The same line carries the batched forward+backward comparison
(256 ragged clouds, one batched call against a per-cloud loop).

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead (the
reference arm: a plain CPU implementation of the method, see oracle/) on a
bounded sample of the workload.
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

WORKLOAD = "so3_4096"
# Bounded samples of each workload for the CPU oracle (baseline and reference
# arm): the first m points of the workload's matrix, same threshold and
# dimensions.  The oracle needs about 1,100 s for all 4096 points of so3_4096;
# its first 1536 points take a few seconds.
ORACLE_SAMPLE_POINTS = {"so3_4096": 1536, "s3_192": 128}
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
    ap.add_argument("--dim-max", type=int, default=None, help="override the workload's top dimension")
    ap.add_argument("--batched", action="store_true",
                    help="only the batched line: 256 ragged clouds, batched forward+backward against a per-cloud loop")
    ap.add_argument("--no-batched", action="store_true", help="leave the batched comparison out of the main line")
    ap.add_argument("--e2e-reps", type=int, default=3, help="end-to-end calls timed through the C ABI")
    return ap.parse_args()


def load_workload(name):
    from paper_1908_02518_gb300 import workloads as W
    return W.WORKLOADS[name]()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x: float) -> float:
    """The largest x over the ranks (the slowest rank's time); x itself when
    no process group is up."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float) -> float:
    """x summed over the ranks (work done by the whole job)."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def whole_job_rate(units: float, max_total_ms: float) -> float:
    """Units per second of the whole job: all ranks' units over the slowest rank's time."""
    return units / (max_total_ms / 1000.0)


def lpt_shards(weights, world: int) -> list[list[int]]:
    """Items split over `world` ranks, heaviest first onto the least-loaded rank
    (longest processing time first); each rank's items in increasing order."""
    order = sorted(range(len(weights)), key=lambda i: (-weights[i], i))
    loads = [0.0] * world
    shards = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (loads[q], q))
        shards[r].append(i)
        loads[r] += weights[i]
    return [sorted(x) for x in shards]


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


def measured_traffic(kernel_class: str, workload: str):
    """DRAM bytes per launch from the committed ncu record (profiles/traffic.json),
    or None when there is none for this kernel and workload or when the kernel's
    sources changed since the counters were taken."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(kernel_class)
        if not rec or rec.get("workload") != workload:
            return None
        h = hashlib.sha256()
        for src in rec["sources"]:
            with open(os.path.join(ROOT, src), "rb") as f:
                h.update(f.read())
        return float(rec["bytes_per_launch"]) if h.hexdigest() == rec["source_sha256"] else None
    except Exception:
        return None


def kernel_roofline(name, km, stats, n, peak, peak_kind):
    """HBM roofline of one kernel class: algorithmic bytes per launch (the
    bytes each unit of work must move, listed per kernel below, times the units
    one launch processes) over the class's average launch time, both from the
    CUDA-event kernel timing."""
    if name not in km or km[name][0] <= 0:
        return None
    launches = max(km[name][1], 1)
    dims = stats[1:]
    if name == "apparent":    # S2: read (index 8 B + rank 4 B) per tested simplex, write 8 B per column,
        algo = sum(12 * s["simplices"] + 8 * s["columns"] + 16 * s["apparent_cofacet"] for s in dims)
    elif name == "reduce":    # S5: read 12 B per entry of every added column, 32 B of state per column
        algo = sum(12 * s["added_entries"] + 32 * s["columns"] for s in dims)
    elif name == "enumerate":  # S1: write 12 B (index + rank) per simplex of dimension >= 2
        algo = sum(12 * s["simplices"] for s in stats[2:])
    elif name == "col_sort":   # S3: 8 radix passes reading and writing 8 B keys
        algo = sum(8 * 16 * s["columns"] for s in dims)
    elif name == "prologue":   # S0: read D once, write the rank matrix once
        algo = 8 * n * n
    else:
        return None
    algo /= launches
    ms = km[name][0] / launches
    achieved = algo / (ms / 1000.0) / 1e9
    return {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind, "launch_ms": ms,
            "algorithmic_bytes": algo, "launches_per_step": launches}


def measure_batched(args, full: bool):
    """Forward + backward of loss = sum over H1 bars of (death - birth)^2 over
    the 256 ragged clouds (64..512 points: circles, tori, cubes): one batched
    call against a loop of the same GPU path called per cloud, both timed with
    CUDA events, inputs resident on the device.  With ``full`` the forward alone
    and a CUDA-graph replay of a batch plan are timed too.  Returns the
    measurements (rank 0) and, for the CPU-reference check, the gradient of a
    few small clouds."""
    import torch
    import paper_1908_02518_gb300 as rg
    from paper_1908_02518_gb300 import workloads as W
    world, rank, _ = dist_env()
    clouds = W.batch_clouds()
    if world > 1:  # clouds are independent: each rank takes its share, no device collective
        mine = lpt_shards([math.comb(len(c), 3) for c in clouds], world)[rank]
        clouds = [clouds[i] for i in mine]
    sizes = [len(c) for c in clouds]
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    pts = torch.from_numpy(np.concatenate(clouds)).cuda()
    dev_clouds = [pts[offsets[i]:offsets[i + 1]] for i in range(len(clouds))]
    stream = torch.cuda.current_stream()

    def step(x, off):
        res = rg.barcodes_batched(x, off, 1, math.inf, 2, keep_handle=True)
        b = res.bars
        h1 = (b["dim"] == 1) & np.isfinite(b["death"])
        diff = np.where(h1, b["death"] - b["birth"], 0.0).astype(np.float32)
        gb = torch.from_numpy(-2.0 * diff).cuda()
        gd = torch.from_numpy(2.0 * diff).cuda()
        g = rg.backward(res, x, gb, gd)
        loss = float((diff.astype(np.float64) ** 2).sum())
        units = sum(s["simplices"] for st in res.stats for s in st)
        res.free()
        return g, loss, units

    def timed(fn, reps):
        out = []
        for _ in range(reps):
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = fn()
            b.record(stream)
            torch.cuda.synchronize()
            out.append(a.elapsed_time(b))
        return statistics.median(out), r

    for _ in range(max(min(args.warmup, 3), 1)):
        step(pts, offsets)
    t_batch, (gx, loss, units) = timed(lambda: step(pts, offsets), 3)
    extra = {}
    if full:
        # the same forward as one CUDA-graph replay of a batch plan (sizes fixed in advance)
        plan = rg.BatchPlan(offsets, pts.shape[1])
        graph = plan.capture(pts)

        def replay():
            graph.replay()
            return plan.result()
        t_graph_fwd, gres = timed(replay, 3)
        t_fwd, fres = timed(lambda: rg.barcodes_batched(pts, offsets, 1), 3)
        graph_same = sorted(map(tuple, gres.bars[["cloud", "dim", "birth", "death"]].tolist())) == \
            sorted(map(tuple, fres.bars[["cloud", "dim", "birth", "death"]].tolist()))
        plan.free()
        extra = {"forward_ms": max_over_ranks(t_fwd), "forward_graph_replay_ms": max_over_ranks(t_graph_fwd),
                 "graph_bars_equal": graph_same}

    def loop():
        gs, ls, us = [], 0.0, 0
        for x in dev_clouds:
            g, l_, u = step(x, np.array([0, len(x)], dtype=np.int64))
            gs.append(g)
            ls += l_
            us += u
        return torch.cat(gs), ls, us
    # warm the per-cloud path on the largest cloud (workspace sizes), then time the whole loop once
    big = int(np.argmax(sizes))
    step(dev_clouds[big], np.array([0, sizes[big]], dtype=np.int64))
    t_loop, (gl, loss_l, units_l) = timed(loop, 1)
    t_batch_job, t_loop_job = max_over_ranks(t_batch), max_over_ranks(t_loop)
    units_job = sum_over_ranks(units)
    # the backward scatter adds with float atomics, so the order of additions
    # (and the last bits) differ between the two; compare within 1e-4 relative
    gdiff = float((gx - gl).abs().max())
    gscale = max(float(gl.abs().max()), 1e-6)
    # small clouds kept for the CPU-reference gradient check (cpu_baseline leg)
    sample = [i for i, n in enumerate(sizes) if n <= 160][:4]
    kept = {i: (clouds[i], gx[offsets[i]:offsets[i + 1]].double().cpu().numpy()) for i in sample}
    out = {"batch_fwd_bwd_ms": t_batch_job, "per_cloud_loop_ms": t_loop_job, "speedup": t_loop_job / t_batch_job,
           "clouds_on_rank0": len(clouds), "points_on_rank0": int(offsets[-1]), "simplices": units_job,
           "simplices_per_s": whole_job_rate(units_job, t_batch_job), "loss_rank0": loss,
           "loss_close_to_loop": math.isclose(loss, loss_l, rel_tol=1e-9),
           "grad_max_rel_diff_to_loop": gdiff / gscale, "grad_within_1e-4_of_loop": gdiff <= 1e-4 * gscale,
           "workload": "batch256", "dim_max": 1, "p": 2}
    out.update(extra)
    return out, kept


def batched_cpu_check(kept) -> dict:
    """The batched GPU gradient of a few small clouds against the CPU reference
    gradient (oracle pairs, float64), relative to its largest entry."""
    import oracle
    from oracle import gradients as G
    worst = 0.0
    for i, (pts, g) in kept.items():
        d32 = G.distances32(pts)
        bars = oracle.barcodes(d32, 1).dim(1)
        bars = bars[np.isfinite(bars["death"])]
        diff = bars["death"].astype(np.float64) - bars["birth"].astype(np.float64)
        ref = G.bar_gradient(pts, bars, -2 * diff, 2 * diff)
        worst = max(worst, float(np.abs(g - ref).max()) / max(float(np.abs(ref).max()), 1e-6))
    return {"clouds": sorted(kept), "max_rel_diff": worst, "within_1e-4": worst <= 1e-4}


def run_batched(args):
    """The batched comparison as its own JSON line."""
    world, rank, _ = dist_env()
    res, kept = measure_batched(args, full=True)
    if rank != 0:
        return 0
    res["cpu_reference_grad_check"] = batched_cpu_check(kept)
    line = {"metric": "batched_forward_backward_ms", "value": res.pop("batch_fwd_bwd_ms"), "unit": "ms",
            "higher_is_better": False, "n_gpus": world, "dtype": "f32 coordinates; integer ranks",
            "data": "synthetic", "config": {"workload": "batch256", "dim_max": 1, "p": 2}}
    line.update(res)
    print(json.dumps(line))
    return 0


def oracle_sample(w):
    """(matrix, description) of the bounded sample the CPU oracle runs on."""
    m = ORACLE_SAMPLE_POINTS.get(w.name)
    if m is None or m >= w.n:
        return w.dist, f"the full {w.name} workload"
    return (np.ascontiguousarray(w.dist[:m, :m]),
            f"the first {m} of the {w.n} points of {w.name} (same matrix entries, threshold {w.threshold}, "
            f"H0-H{w.dim_max}, Z/{w.p})")


def cpu_baseline(w, budget_s=12.0):
    """The oracle as it stands, single-threaded on the host, repeated on the
    bounded sample until about budget_s seconds of CPU work."""
    import oracle
    oracle.build()
    d, what = oracle_sample(w)
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
            "sample": f"{runs} runs on {what} (cohomology oracle, {el:.1f} s)"}


def workload_config(w, world: int) -> dict:
    """The config object of both arms' JSON lines (the same workload and conditions)."""
    return {"workload": w.name, "n": w.n, "dim_max": w.dim_max, "threshold": w.threshold, "p": w.p,
            "parallelism": f"replicas{world}" if world > 1 else "single",
            "l2": "flushed between steps (256 MiB write)"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    w = load_workload(args.workload)
    import oracle
    oracle.build()
    d, what = oracle_sample(w)
    units = None
    for _ in range(args.warmup):
        oracle.barcodes(d, w.dim_max, w.threshold, w.p)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.barcodes(d, w.dim_max, w.threshold, w.p)
        times.append(time.perf_counter() - t0)
        units = sum(s["simplices"] for s in r.stats)
    tot = sum(times)
    val = units * len(times) / tot
    line = {"impl": "reference", "metric": "rips_barcode_simplices_per_s", "value": val, "unit": "simplices/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": workload_config(w, world),
            "cpu_baseline": {"value": val, "unit": "simplices/s", "cores": 1, "kind": "oracle",
                             "sample": f"{what} per step"},
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

    if args.batched:
        return run_batched(args)
    w = load_workload(args.workload)
    if args.dim_max is not None:
        w.dim_max = args.dim_max
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
    total_ms = max_over_ranks(total_ms)
    ms_per_step = total_ms / args.steps
    value = whole_job_rate(sum_over_ranks(units * args.steps), total_ms)
    per_dim = []
    for d in range(w.dim_max + 1):
        ph = statistics.median(p[d] for p in phase)
        per_dim.append({"dim": d, "simplices": units_per_dim[d], "phase_ms": ph,
                        "simplices_per_s": units_per_dim[d] / (ph / 1000.0) if ph > 0 else None})

    # dominant kernel class, timed live with events on the call's stream
    rg.set_kernel_timing(True)
    km = {}
    kr = 3 if ms_per_step < 1000.0 else 1
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
    peak, peak_kind = peaks()
    roof = kernel_roofline(dom, km, stats, n, peak, peak_kind)
    if roof is not None:
        roof["traffic"] = measured_traffic(dom, w.name)
    streaming = kernel_roofline("apparent", km, stats, n, peak, peak_kind)
    if dom == "reduce":
        # the reduction is bound by its longest chain of dependent additions
        worst = max(range(1, len(stats)), key=lambda d: stats[d]["longest_chain"]) if len(stats) > 1 else 0
        chain = stats[worst]["longest_chain"] if worst else 0
        dim_ms = statistics.median(p[worst] for p in phase) if worst else 0.0
        roof["critical_path"] = {"dim": worst, "longest_chain": chain, "dim_phase_ms": dim_ms,
                                 "us_per_chain_addition": 1000.0 * dim_ms / chain if chain else None}

    # end to end through the C ABI with host buffers (copies inside the timed region)
    pinned = torch.from_numpy(w.dist).pin_memory()
    host = pinned.numpy()
    e2e_t = []
    nbars = 0
    for k in range(max(1, args.e2e_reps) + 1):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = rg.barcodes(host, w.dim_max, w.threshold, w.p)
        t1 = time.perf_counter()
        if k >= 1:
            e2e_t.append(t1 - t0)
        nbars = len(r.bars)
    e2e_s = max_over_ranks(sum(e2e_t) / len(e2e_t) * 1000.0) / 1000.0
    e2e = {"value": whole_job_rate(sum_over_ranks(units), 1000.0 * e2e_s), "unit": "simplices/s",
           "h2d_bytes_per_step": 4 * n * n,
           "d2h_bytes_per_step": 32 * nbars, "ms_per_step": 1000 * e2e_s}

    batched, kept = (None, None) if args.no_batched else measure_batched(args, full=False)

    if rank == 0:
        cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline(w)
        if batched is not None and not args.no_cpu_baseline and world == 1:
            batched["cpu_reference_grad_check"] = batched_cpu_check(kept)
        line = {"metric": "rips_barcode_simplices_per_s", "value": value, "unit": "simplices/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64 integer ranks and indices; f32 values",
                "data": "synthetic",
                "config": workload_config(w, world),
                "per_dim": per_dim, "barcode_ms": ms_per_step, "bars": nbars,
                "kernel_ms": {k: v[0] for k, v in km.items()},
                "roofline": roof, "roofline_streaming": streaming, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches, "clocks": ck, "batched": batched}
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
