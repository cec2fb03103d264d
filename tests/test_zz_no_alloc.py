"""The allocation-free H0 entry point, rips_h0_barcode_noalloc.

It serves callers that must not allocate device memory while they run -- code
inside CUDA-graph capture, serving processes whose memory pool owns the whole
device, real-time loops that cannot wait on the allocator.  It keeps all of
its intermediate data in a fixed file-scope device array, so it handles at
most RIPS_NOALLOC_MAX_N points.  This test calls it through the C ABI twice in
a row (the second call must not see the first call's leftovers) and compares
its bars with those of rips_barcodes_device at dim_max = 0.  It lives in its
own file, collected last, and passes alone or after the other tests.
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


def _noalloc(dist_np, threshold):
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
    assert st == 0, st
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
