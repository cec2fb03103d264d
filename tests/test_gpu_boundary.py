"""The batched distance-matrix entry point and the distance-only backward,
through the C ABI, against the CPU oracle.

rips_barcodes_batched_dists takes one device matrix per cloud (any finite
metric, not only Euclidean point clouds): every cloud's bars must equal the
oracle's bar by bar, simplex indices included.  rips_barcodes_backward_dist
must put dL/dbirth and dL/ddeath on the critical edge of each bar's simplex,
which the CPU reference (oracle/gradients.py) derives from the oracle's pairs.
"""
import math

import numpy as np
import pytest

from paper_1908_02518_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U64MAX = int(np.iinfo(np.uint64).max)


def _key(bars, cloud=None):
    out = []
    for b in bars:
        if cloud is not None and int(b["cloud"]) != cloud:
            continue
        ds = int(b["death_simplex"])
        out.append((int(b["dim"]), float(b["birth"]), float(b["death"]), int(b["birth_simplex"]),
                    U64MAX if ds < 0 else ds))
    return sorted(out)


def _mats():
    rng = np.random.Generator(np.random.PCG64(5150))
    return [W.distance_matrix(W.torus_points(90, 51)),
            W.random_integer_matrix(23, 52, levels=4),          # not Euclidean, many ties
            W.distance_matrix(rng.random((57, 3)).astype(np.float32)),
            W.distance_matrix(W.sphere_points(40, 53))]


@pytest.mark.parametrize("p,t", [(2, math.inf), (3, math.inf), (2, 0.9)])
def test_batched_dists_matches_oracle(oracle_mod, p, t):
    import torch
    import paper_1908_02518_gb300 as rg
    mats = _mats()
    res = rg.barcodes_batched_dists([torch.from_numpy(m).cuda() for m in mats], 2, t, p)
    assert res.clouds == len(mats)
    for c, m in enumerate(mats):
        want = oracle_mod.barcodes(m, 2, t, p)
        assert res.thresholds[c] == want.threshold
        assert _key(res.bars, c) == _key(want.bars), c


def test_backward_dist_matches_reference(oracle_mod):
    import torch
    import paper_1908_02518_gb300 as rg
    from oracle import gradients as G
    mats = _mats()
    dev = [torch.from_numpy(m).cuda() for m in mats]
    res = rg.barcodes_batched_dists(dev, 1, keep_handle=True)
    nb = len(res.bars)
    gb = torch.linspace(-1.0, 1.0, nb, dtype=torch.float32, device="cuda")
    gd = torch.linspace(0.5, 2.0, nb, dtype=torch.float32, device="cuda")
    grads = rg.backward_dist(res, dev, gb, gd)
    gbh, gdh = gb.cpu().numpy(), gd.cpu().numpy()
    for c, m in enumerate(mats):
        want = np.zeros(m.shape, dtype=np.float64)
        for q, b in enumerate(res.bars):
            if int(b["cloud"]) != c:
                continue
            dim = int(b["dim"])
            if dim >= 1:
                want[G.critical_edge(m, int(b["birth_simplex"]), dim)] += gbh[q]
            if np.isfinite(b["death"]):
                want[G.critical_edge(m, int(b["death_simplex"]), dim + 1)] += gdh[q]
        np.testing.assert_allclose(grads[c].cpu().numpy(), want, rtol=1e-5, atol=1e-5)
    res.free()


def test_backward_dist_equals_points_backward_grad_dist():
    """On a Euclidean cloud both backward entry points give the same dL/dD."""
    import torch
    import paper_1908_02518_gb300 as rg
    pts = W.torus_points(70, 54)
    x = torch.from_numpy(pts).cuda()
    d = rg.distance_matrix(x)
    res = rg.barcodes(d, 1, keep_handle=True)
    nb = len(res.bars)
    gb = torch.linspace(-1.0, 1.0, nb, dtype=torch.float32, device="cuda")
    gd = torch.linspace(0.5, 2.0, nb, dtype=torch.float32, device="cuda")
    (g1,) = rg.backward_dist(res, [d], gb, gd)
    g2 = torch.zeros(70 * 70, dtype=torch.float32, device="cuda")
    rg.backward(res, x, gb, gd, grad_dist=g2)
    np.testing.assert_allclose(g1.cpu().numpy().ravel(), g2.cpu().numpy(), rtol=1e-6, atol=1e-6)
    res.free()


@pytest.mark.parametrize("layout", ["lower", "upper"])
def test_packed_triangle_matches_oracle(oracle_mod, layout):
    """The packed lower / upper triangle input formats give the oracle's bars of
    the full matrix, bar by bar."""
    import paper_1908_02518_gb300 as rg
    for d, t, p in [(W.distance_matrix(W.torus_points(120, 61)), 1.2, 2), (W.random_integer_matrix(25, 62), math.inf, 3)]:
        n = d.shape[0]
        if layout == "lower":
            packed = np.concatenate([d[i, :i] for i in range(1, n)])
        else:
            packed = np.concatenate([d[i, i + 1:] for i in range(n - 1)])
        got = rg.barcodes_packed(packed.astype(np.float32), n, layout, 2, t, p)
        want = oracle_mod.barcodes(d, 2, t, p)
        assert _key(got.bars) == _key(want.bars)
