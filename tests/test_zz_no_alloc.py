"""The allocation-free H0 entry point, rips_h0_barcode_noalloc.

It serves callers that must not allocate device memory while they run -- a
serving process whose memory pool owns the whole device, a real-time loop that
cannot wait on cudaMalloc / cudaFree.  It keeps all of its intermediate data in
a fixed file-scope device array, so it handles at most RIPS_NOALLOC_MAX_N
points.  These tests call it through the C ABI several times in a row (a call
must not see an earlier call's leftovers) and compare its bars with those of
rips_barcodes_device at dim_max = 0 and with the CPU oracle, simplex indices
included, from one point up to the maximum size and on both paths of the edge
sort (one block up to 8192 edges, radix passes beyond).  The file is collected
last and passes alone or after the other tests.
"""
import ctypes as C
import math

import numpy as np
import pytest

from paper_1908_02518_gb300 import workloads as W

pytestmark = pytest.mark.gpu

MAX_N = 512


def _sorted_bars(arr):
    return sorted((int(b["dim"]), float(b["birth"]), float(b["death"]), int(b["birth_simplex"]),
                   int(b["death_simplex"])) for b in arr)


def _noalloc(dist_np, threshold, expect=0):
    import torch
    import paper_1908_02518_gb300 as rg
    from paper_1908_02518_gb300 import _lib
    lib = _lib.load()
    n = dist_np.shape[0]
    d = torch.from_numpy(np.ascontiguousarray(dist_np)).cuda()
    bars = torch.zeros(n * 32, dtype=torch.uint8, device="cuda")   # room for n bars of 32 bytes
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    st = lib.rips_h0_barcode_noalloc(C.c_void_p(d.data_ptr()), n, C.c_float(threshold),
                                     C.c_void_p(bars.data_ptr()), C.c_void_p(count.data_ptr()), C.c_void_p(stream))
    assert st == expect, st
    if expect != 0:
        return None
    torch.cuda.synchronize()
    k = int(count.item())
    raw = bars.cpu().numpy()[: k * 32].tobytes()
    return np.frombuffer(raw, dtype=rg.BAR_DTYPE)


def test_noalloc_matches_barcodes_device_twice():
    import torch
    import paper_1908_02518_gb300 as rg
    cases = [(W.distance_matrix(W.torus_points(300, 11)), 1.2),
             (W.distance_matrix(W.cube_points(MAX_N, 12)), math.inf)]
    for dist, t in cases:  # two calls in a row on different inputs
        got = _noalloc(dist, t)
        want = rg.barcodes(torch.from_numpy(dist).cuda(), 0, t, 2)
        assert _sorted_bars(got) == _sorted_bars(want.bars)


def test_noalloc_rejects_too_many_points():
    import torch
    from paper_1908_02518_gb300 import _lib
    lib = _lib.load()
    n = MAX_N + 1
    d = torch.zeros((n, n), dtype=torch.float32, device="cuda")
    bars = torch.zeros(n * 32, dtype=torch.uint8, device="cuda")
    count = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = lib.rips_h0_barcode_noalloc(C.c_void_p(d.data_ptr()), n, C.c_float(1.0), C.c_void_p(bars.data_ptr()),
                                     C.c_void_p(count.data_ptr()), None)
    assert st == -1


def test_noalloc_matches_oracle_small_sizes(oracle_mod):
    """n = 1, 2, 64 (single-block sort) and 300, each against the oracle's
    Kruskal bars, simplex indices included; the calls run back to back."""
    cases = [(np.zeros((1, 1), dtype=np.float32), math.inf),
             (W.distance_matrix(W.cube_points(2, 31)), math.inf),
             (W.distance_matrix(W.torus_points(64, 32)), 1.0),
             (W.distance_matrix(W.torus_points(64, 33)), math.inf),
             (W.distance_matrix(W.cube_points(300, 34)), 0.2)]
    for dist, t in cases:
        got = _noalloc(dist, t)
        want = oracle_mod.barcodes(dist, 0, t, 2)
        assert _sorted_bars(got) == sorted(
            (int(b["dim"]), float(b["birth"]), float(b["death"]), int(b["birth_simplex"]),
             int(b["death_simplex"]) if np.isfinite(b["death"]) else 2 ** 64 - 1) for b in want.bars), dist.shape


def test_noalloc_rejects_nan_then_recovers():
    import torch
    import paper_1908_02518_gb300 as rg
    dist = W.distance_matrix(W.cube_points(40, 35))
    bad = dist.copy()
    bad[7, 3] = np.nan
    _noalloc(bad, math.inf, expect=-1)
    got = _noalloc(dist, math.inf)
    want = rg.barcodes(torch.from_numpy(dist).cuda(), 0, math.inf, 2)
    assert _sorted_bars(got) == _sorted_bars(want.bars)
