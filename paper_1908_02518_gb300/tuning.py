"""Launch-parameter tuning per (dimension, cloud size), and the autotuner.

The library looks its launch and scheduling parameters up per dimension and
per the largest cloud size of a call (``rips_tuning_t`` in include/rips.h):
how many additions a warp makes on one column before a block takes it over,
the largest merge a warp makes, and blocks per SM of the reduction and of the
enumeration / test kernels.  None of them changes a result.  ``autotune`` times
candidate settings on caller-supplied inputs and installs, for every dimension
and cloud-size bucket, the fastest one; ``save`` / ``load`` keep the table as
JSON.
"""
from __future__ import annotations

import ctypes as C
import itertools
import json
import math
import time

from . import _lib

DEFAULT = {"warp_chain_limit": 32, "warp_merge_max": 2048, "reduce_blocks_per_sm": 0, "scan_blocks_per_sm": 16}
FIELDS = tuple(DEFAULT)

# the candidate grid the autotuner walks (the default is part of it)
CANDIDATES = {
    "warp_chain_limit": (8, 32, 128),
    "warp_merge_max": (512, 2048, 8192),
    "reduce_blocks_per_sm": (0, 1),
    "scan_blocks_per_sm": (8, 16, 32),
}


def set_tuning(dim: int, n_lo: int, n_hi: int, params: dict) -> None:
    """Use ``params`` for dimension ``dim`` when the largest cloud has n_lo..n_hi points."""
    full = dict(DEFAULT, **params)
    t = _lib.Tuning(*(int(full[f]) for f in FIELDS))
    _lib.check(_lib.load().rips_set_tuning(dim, n_lo, n_hi, C.byref(t)), "rips_set_tuning")


def get_tuning(dim: int, n: int) -> dict:
    t = _lib.Tuning()
    _lib.check(_lib.load().rips_get_tuning(dim, n, C.byref(t)), "rips_get_tuning")
    return {f: int(getattr(t, f)) for f in FIELDS}


def clear_tuning() -> None:
    _lib.load().rips_clear_tuning()


def bucket(n: int) -> tuple[int, int]:
    """Cloud-size bucket of n: powers of two, [2^k + 1, 2^(k+1)]."""
    hi = 1 << max(0, math.ceil(math.log2(max(n, 1))))
    return (hi // 2 + 1 if hi > 1 else 1, hi)


def _phase_times(run, reps: int) -> list[float]:
    """Median per-dimension phase times (ms) of ``run()`` over ``reps`` calls."""
    rows = []
    for _ in range(reps):
        res = run()
        rows.append(res.phase_ms)
    return [sorted(r[d] for r in rows)[len(rows) // 2] for d in range(len(rows[0]))]


def autotune(run, n_max: int, dims, reps: int = 3, grid: dict | None = None, budget_s: float = 60.0) -> dict:
    """Time every candidate setting on ``run()`` (a callable making one barcode
    call, e.g. ``lambda: barcodes_batched(points, offsets, 1)``, whose largest
    cloud has ``n_max`` points) and install, for each dimension in ``dims``, the
    setting with the smallest median phase time for that dimension in n_max's
    bucket.  Stops trying new candidates after ``budget_s`` seconds.  Returns
    {dim: {"params": ..., "ms": ..., "default_ms": ...}}."""
    grid = grid or CANDIDATES
    lo, hi = bucket(n_max)
    dims = list(dims)
    cands = [dict(zip(FIELDS, v)) for v in itertools.product(*(grid[f] for f in FIELDS))]
    cands.sort(key=lambda c: c != DEFAULT)  # the default first: it is the baseline
    best = {}
    t_end = time.time() + budget_s
    for c in cands:
        if best and time.time() > t_end:
            break
        for d in dims:
            set_tuning(d, lo, hi, c)
        run()  # warm-up (buffers sized, clocks up)
        ms = _phase_times(run, reps)
        for d in dims:
            if d not in best or ms[d] < best[d]["ms"]:
                best[d] = {"params": dict(c), "ms": ms[d], "default_ms": best.get(d, {}).get("default_ms", ms[d])}
    for d in dims:
        set_tuning(d, lo, hi, best[d]["params"])
    return {d: dict(v, bucket=[lo, hi]) for d, v in best.items()}


def save(table: dict, path: str) -> None:
    with open(path, "w") as f:
        json.dump({str(d): v for d, v in table.items()}, f, indent=1)


def load(path: str) -> dict:
    """Install a table written by ``save``."""
    with open(path) as f:
        table = {int(d): v for d, v in json.load(f).items()}
    for d, v in table.items():
        set_tuning(d, v["bucket"][0], v["bucket"][1], v["params"])
    return table
