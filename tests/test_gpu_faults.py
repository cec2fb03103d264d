"""Failure detection without faulting the GPU.

Every wait in the library's kernels is bounded and every capacity is checked,
so the failures a caller can meet come back as status codes and leave the
context usable.  These tests inject them through rips_set_limits: a grid-barrier
wait and a chain of additions that give up almost at once (a timeout status), a
pivot table far too small (out of memory), and a reduction arena too small to
start with (grown and the dimension redone: same bars).  After each, a call with
the default limits must give the right barcode.
"""
import math

import pytest

from paper_1908_02518_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _default_limits():
    import paper_1908_02518_gb300 as rg
    rg.set_limits()
    yield
    rg.set_limits()


def _bars(res):
    b = res.bars
    return sorted(zip(b["dim"].tolist(), b["birth"].tolist(), b["death"].tolist(), b["birth_simplex"].tolist(),
                      b["death_simplex"].tolist()))


def _s3(n):
    import torch
    return torch.from_numpy(W.distance_matrix(W.sphere_points(n, 1005, 4))).cuda()


def test_waits_that_run_out_return_a_timeout_status():
    import paper_1908_02518_gb300 as rg
    from paper_1908_02518_gb300 import _lib
    d = _s3(96)  # dimension 3 holds a chain of about 3500 additions
    want = _bars(rg.barcodes(d, 3, math.inf, 3))
    rg.set_limits(barrier_wait_ns=1000, chain_ns=1000)
    with pytest.raises(_lib.RipsError) as e:
        rg.barcodes(d, 3, math.inf, 3)
    assert e.value.status == -6  # RIPS_ERR_DEVICE_TIMEOUT
    rg.set_limits()
    assert _bars(rg.barcodes(d, 3, math.inf, 3)) == want


def test_a_full_pivot_table_is_reported_as_out_of_memory():
    import paper_1908_02518_gb300 as rg
    from paper_1908_02518_gb300 import _lib
    d = _s3(48)
    want = _bars(rg.barcodes(d, 3, math.inf, 3))
    rg.set_limits(table_slots=16)
    with pytest.raises(_lib.RipsError) as e:
        rg.barcodes(d, 3, math.inf, 3)
    assert e.value.status == -4  # RIPS_ERR_OOM
    rg.set_limits()
    assert _bars(rg.barcodes(d, 3, math.inf, 3)) == want


def test_a_tiny_arena_is_grown_and_gives_the_same_bars():
    import torch
    import paper_1908_02518_gb300 as rg
    d = torch.from_numpy(W.distance_matrix(W.torus_points(300, 21))).cuda()
    want = _bars(rg.barcodes(d, 2, 1.2, 2))
    rg.set_limits(arena_entries=256)
    assert _bars(rg.barcodes(d, 2, 1.2, 2)) == want
