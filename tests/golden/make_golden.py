"""Writes the expected barcodes of the full-size workloads, computed by the CPU
oracle only (oracle/, cohomology method).  Run from the repository root:

    python tests/golden/make_golden.py [workload ...]

Each workload gives tests/golden/<name>.bars.txt.gz (the batched workload:
batch256.bars.txt.gz, one header per cloud): a header with the SHA-256 of
the FP32 distance matrix (so a test can check that its input is bit-identical)
and one line per bar: dim birth_bits death_bits birth_simplex death_simplex
(float bits in hex, death_simplex -1 for essential classes), plus the oracle's
per-dimension counts.
"""
from __future__ import annotations

import gzip
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1908_02518_gb300 import workloads as W  # noqa: E402


def write(name, dist, dim_max, threshold, p, extra=None):
    t0 = time.time()
    r = oracle.barcodes(dist, dim_max, threshold, p, method="coh")
    el = time.time() - t0
    path = os.path.join(HERE, f"{name}.bars.txt.gz")
    head = {"workload": name, "sha256": W.matrix_digest(dist), "n": int(dist.shape[0]), "dim_max": dim_max,
            "threshold": threshold, "p": p, "threshold_used": r.threshold, "stats": r.stats,
            "oracle_seconds": round(el, 2), "source": "oracle/ (cohomology method), tests/golden/make_golden.py"}
    if extra:
        head.update(extra)
    with gzip.open(path, "wt") as f:
        f.write("# " + json.dumps(head) + "\n")
        for b in r.bars:
            f.write(f"{int(b['dim'])} {np.float32(b['birth']).view(np.uint32):08x} "
                    f"{np.float32(b['death']).view(np.uint32):08x} {int(b['birth_simplex'])} "
                    f"{int(b['death_simplex'])}\n")
    print(f"{name}: {len(r.bars)} bars, oracle {el:.1f} s -> {path}")


def read(path):
    """(header, bars) with bars a list of (dim, birth, death, birth_simplex, death_simplex)."""
    with gzip.open(path, "rt") as f:
        head = json.loads(f.readline()[2:])
        bars = []
        for line in f:
            d, b, e, bs, ds = line.split()
            bars.append((int(d), float(np.uint32(int(b, 16)).view(np.float32)),
                         float(np.uint32(int(e, 16)).view(np.float32)), int(bs), int(ds)))
    return head, bars


def bar_line(dim, birth, death, bs, ds):
    return (f"{int(dim)} {np.float32(birth).view(np.uint32):08x} {np.float32(death).view(np.uint32):08x} "
            f"{int(bs)} {int(ds)}")


def canonical_digest(bars):
    """SHA-256 of the bars (dim, birth, death, birth_simplex, death_simplex; -1 for
    an essential death simplex) sorted as tuples, one bar_line per bar."""
    import hashlib
    h = hashlib.sha256()
    for t in sorted(bars):
        h.update((bar_line(*t) + "\n").encode())
    return h.hexdigest()


def batch():
    """All 256 clouds of the batched workload in one file: per cloud a header line
    ('#' + JSON with its matrix digest, the H0 bar count and the digest of its H0
    bars) followed by its H1 bars in full."""
    clouds = W.batch_clouds()
    path = os.path.join(HERE, "batch256.bars.txt.gz")
    t0 = time.time()
    with gzip.open(path, "wt") as f:
        for c, pts in enumerate(clouds):
            d = W.distance_matrix(pts)
            r = oracle.barcodes(d, 1, float("inf"), 2, method="coh")
            tup = [(int(b["dim"]), float(b["birth"]), float(b["death"]), int(b["birth_simplex"]),
                    int(b["death_simplex"])) for b in r.bars]
            h0 = [t for t in tup if t[0] == 0]
            head = {"cloud": c, "sha256": W.matrix_digest(d), "n": int(d.shape[0]), "threshold_used": r.threshold,
                    "stats": r.stats, "h0_count": len(h0), "h0_digest": canonical_digest(h0)}
            f.write("# " + json.dumps(head) + "\n")
            for t in tup:
                if t[0] == 1:
                    f.write(bar_line(*t) + "\n")
    print(f"batch: {len(clouds)} clouds, oracle {time.time() - t0:.1f} s -> {path}")


def read_batch(path):
    """list of (header, H1 bars) per cloud"""
    out = []
    with gzip.open(path, "rt") as f:
        for line in f:
            if line.startswith("# "):
                out.append((json.loads(line[2:]), []))
                continue
            d, b, e, bs, ds = line.split()
            out[-1][1].append((int(d), float(np.uint32(int(b, 16)).view(np.float32)),
                               float(np.uint32(int(e, 16)).view(np.float32)), int(bs), int(ds)))
    return out


def main(names):
    for name in names:
        if name == "batch":
            batch()
            continue
        w = W.WORKLOADS[name]()
        write(name, w.dist, w.dim_max, w.threshold, w.p)


if __name__ == "__main__":
    main(sys.argv[1:] or ["cube100", "torus1000", "so3_4096", "s3_192", "clifford1500", "batch"])
