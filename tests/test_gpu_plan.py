"""Batch plans: the H0-H1 barcodes of a batch with fixed cloud sizes, every
launch enqueued without host synchronisation, so the forward can be captured
into a CUDA graph and replayed on new coordinates."""
import math

import numpy as np
import pytest

from paper_1908_02518_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ARENA = 1 << 29  # entries; enough for these batches (the default scales with the edge count)


def _bars(res):
    b = res.bars
    return sorted(zip(b["cloud"].tolist(), b["dim"].tolist(), b["birth"].tolist(), b["death"].tolist(),
                      b["birth_simplex"].tolist(), b["death_simplex"].tolist()))


def _batch(count, seed_shift=0):
    clouds = W.batch_clouds(count=count, cloud_seed=40000 + seed_shift)
    offsets = np.concatenate([[0], np.cumsum([len(c) for c in clouds])]).astype(np.int64)
    return np.concatenate(clouds), offsets


def test_plan_matches_the_batched_call():
    import torch
    import paper_1908_02518_gb300 as rg
    pts_np, off = _batch(24)
    pts = torch.from_numpy(pts_np).cuda()
    want = rg.barcodes_batched(pts, off, 1)
    plan = rg.BatchPlan(off, 3, arena_entries=ARENA)
    plan.run(pts)
    got = plan.result()
    assert _bars(got) == _bars(want)
    assert [s[1]["pairs"] for s in got.stats] == [s[1]["pairs"] for s in want.stats]
    plan.free()


def test_captured_graph_replays_on_new_coordinates():
    import torch
    import paper_1908_02518_gb300 as rg
    a_np, off = _batch(16)
    pts = torch.from_numpy(a_np).cuda()
    plan = rg.BatchPlan(off, 3, arena_entries=ARENA)
    g = plan.capture(pts)
    for shift in (0, 7):  # same sizes, other clouds: the graph's launches are fixed, the data not
        b_np, off_b = _batch(16, 0)
        if shift:
            rng = np.random.Generator(np.random.PCG64(shift))
            b_np = (b_np + rng.normal(0, 0.01, b_np.shape)).astype(np.float32)
        assert np.array_equal(off_b, off)
        pts.copy_(torch.from_numpy(b_np))
        g.replay()
        got = plan.result()
        want = rg.barcodes_batched(torch.from_numpy(b_np).cuda(), off, 1)
        assert _bars(got) == _bars(want)
    plan.free()


def test_plan_result_feeds_the_backward():
    import torch
    import paper_1908_02518_gb300 as rg
    pts_np, off = _batch(8)
    pts = torch.from_numpy(pts_np).cuda()
    plan = rg.BatchPlan(off, 3, arena_entries=ARENA)
    plan.run(pts)
    res = plan.result(keep_handle=True)
    ref = rg.barcodes_batched(pts, off, 1, keep_handle=True)
    b = res.bars
    h1 = (b["dim"] == 1) & np.isfinite(b["death"])
    diff = np.where(h1, b["death"] - b["birth"], 0.0).astype(np.float32)
    g1 = rg.backward(res, pts, torch.from_numpy(-2 * diff).cuda(), torch.from_numpy(2 * diff).cuda())
    g2 = rg.backward(ref, pts, torch.from_numpy(-2 * diff).cuda(), torch.from_numpy(2 * diff).cuda())
    assert float((g1 - g2).abs().max()) <= 1e-4 * max(float(g2.abs().max()), 1e-6)
    plan.free()


def test_plan_rejects_bad_arguments():
    import paper_1908_02518_gb300 as rg
    from paper_1908_02518_gb300 import _lib
    with pytest.raises(_lib.RipsError):
        rg.BatchPlan([0, 5, 5], 3)  # an empty cloud
    with pytest.raises(_lib.RipsError):
        rg.BatchPlan([0, 5, 9], 3, p=4)
