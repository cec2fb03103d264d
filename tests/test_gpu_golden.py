"""Full-size parity: the CUDA path against the oracle's stored barcodes of the
five workloads (tests/golden/*.bars.txt.gz, written by
tests/golden/make_golden.py from oracle/ only).  The input matrix's SHA-256 is
checked first, so a difference cannot come from the input generator."""
import math
import os

import numpy as np
import pytest

from paper_1908_02518_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
U64MAX = int(np.iinfo(np.uint64).max)


def _mg():
    import importlib.util
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLD, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    return mg


def _read(name):
    path = os.path.join(GOLD, f"{name}.bars.txt.gz")
    if not os.path.exists(path):
        pytest.skip(f"golden file {name} not generated")
    return _mg().read(path)


def _key_gpu(bars):
    return sorted((int(b["dim"]), float(b["birth"]), float(b["death"]), int(b["birth_simplex"]),
                   int(b["death_simplex"])) for b in bars)


def _key_gold(bars):
    return sorted((d, b, e, bs, U64MAX if ds < 0 else ds) for d, b, e, bs, ds in bars)


@pytest.mark.parametrize("name", ["cube100", "torus1000", "s3_192", "so3_4096"])
def test_workload_matches_golden(name):
    import torch
    import paper_1908_02518_gb300 as rg
    head, bars = _read(name)
    w = W.WORKLOADS[name]()
    assert W.matrix_digest(w.dist) == head["sha256"], "input generator is not bit-identical on this host"
    res = rg.barcodes(torch.from_numpy(w.dist).cuda(), w.dim_max, w.threshold, w.p)
    assert res.threshold == head["threshold_used"]
    g, want = _key_gpu(res.bars), _key_gold(bars)
    if g != want:
        gs, ws = set(g), set(want)
        raise AssertionError(f"{len(g)} vs {len(want)}; only gpu {sorted(gs - ws)[:5]}; only oracle {sorted(ws - gs)[:5]}")
    for d in range(w.dim_max + 1):
        s, o = res.stats[0][d], head["stats"][d]
        assert s["simplices"] == o["simplices"]
        assert s["essential"] == o["essential"]
        if d:
            assert s["pairs"] + s["apparent_cofacet"] == o["pairs"]


def test_batch_matches_golden():
    import torch
    import paper_1908_02518_gb300 as rg
    clouds = W.batch_clouds()
    off = np.concatenate([[0], np.cumsum([c.shape[0] for c in clouds])])
    x = torch.from_numpy(np.concatenate(clouds)).cuda()
    res = rg.barcodes_batched(x, off, dim_max=1)
    path = os.path.join(GOLD, "batch256.bars.txt.gz")
    if not os.path.exists(path):
        pytest.skip("golden file batch256 not generated")
    mg = _mg()
    gold = mg.read_batch(path)
    assert len(gold) == len(clouds)
    for c, pts in enumerate(clouds):
        head, h1 = gold[c]
        assert W.matrix_digest(W.distance_matrix(pts)) == head["sha256"]
        assert _key_gpu(res.dim(1, c)) == _key_gold(h1), c
        h0 = [(d, b, e, bs, -1 if ds == U64MAX else ds) for d, b, e, bs, ds in _key_gpu(res.dim(0, c))]
        assert len(h0) == head["h0_count"], c
        assert mg.canonical_digest(h0) == head["h0_digest"], c


def _gold_batch():
    path = os.path.join(GOLD, "batch256.bars.txt.gz")
    if not os.path.exists(path):
        pytest.skip("golden file batch256 not generated")
    return _mg().read_batch(path)


def test_batch_plan_graph_replay_matches_golden():
    """The CUDA-graph replay of a batch plan over all 256 clouds against the
    oracle's stored barcodes (H1 bar by bar, H0 by count and digest)."""
    import torch
    import paper_1908_02518_gb300 as rg
    clouds = W.batch_clouds()
    off = np.concatenate([[0], np.cumsum([c.shape[0] for c in clouds])]).astype(np.int64)
    gold = _gold_batch()
    mg = _mg()
    x = torch.from_numpy(np.concatenate(clouds)).cuda()
    plan = rg.BatchPlan(off, 3)
    graph = plan.capture(x)
    graph.replay()
    res = plan.result()
    for c in range(len(clouds)):
        head, h1 = gold[c]
        assert _key_gpu(res.dim(1, c)) == _key_gold(h1), c
        h0 = [(d, b, e, bs, -1 if ds == U64MAX else ds) for d, b, e, bs, ds in _key_gpu(res.dim(0, c))]
        assert len(h0) == head["h0_count"], c
        assert mg.canonical_digest(h0) == head["h0_digest"], c
    plan.free()


def test_batch_gradient_matches_cpu_reference():
    """Forward + backward of loss = sum over H1 bars of (death - birth)^2 on all
    256 clouds in one batched call; every cloud's gradient against the CPU
    reference gradient (oracle/gradients.py) on the oracle's stored pairs,
    ||g - g_ref||_inf <= 1e-4 max(||g_ref||_inf, 1e-6)."""
    import torch
    import paper_1908_02518_gb300 as rg
    from oracle import gradients as G
    clouds = W.batch_clouds()
    off = np.concatenate([[0], np.cumsum([c.shape[0] for c in clouds])]).astype(np.int64)
    gold = _gold_batch()
    x = torch.from_numpy(np.concatenate(clouds)).cuda().requires_grad_(True)
    birth, death, dim, cloud = rg.RipsBarcodes.apply(x, off.tolist(), 1)
    fin = torch.isfinite(death) & (dim == 1)
    ((death - birth)[fin] ** 2).sum().backward()
    g = x.grad.double().cpu().numpy()
    dt = np.dtype([("dim", "i4"), ("birth", "f4"), ("death", "f4"), ("birth_simplex", "i8"), ("death_simplex", "i8")])
    for c, pts in enumerate(clouds):
        _, h1 = gold[c]
        bars = np.array([(d, b, e, bs, ds) for d, b, e, bs, ds in h1 if ds >= 0], dtype=dt)
        diff = bars["death"].astype(np.float64) - bars["birth"].astype(np.float64)
        ref = G.bar_gradient(pts, bars, -2 * diff, 2 * diff)
        gc = g[off[c]:off[c + 1]]
        err = np.abs(gc - ref).max() if len(ref) else 0.0
        assert err <= 1e-4 * max(np.abs(ref).max() if len(ref) else 0.0, 1e-6), (c, err)
