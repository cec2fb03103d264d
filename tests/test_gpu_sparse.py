"""The sparse-input path (rips_barcodes_sparse, rips_barcodes_sparse_points):
edges only, rank lookups in the sorted neighbour lists, no n x n array.

* the Clifford torus of 1500 points in R^4 (the paper's torus4 data set at a
  smaller size), threshold 0.4, H0-H2: bar by bar against the oracle's stored
  barcode (tests/golden/clifford1500.bars.txt.gz);
* (i, j, length) lists taken from dense matrices, thresholds, ties and Z/3:
  bar by bar against the oracle on the full matrix;
* the sparse and the dense path agree on the same inputs, statistics included;
* the torus4 size itself, 50,000 points at t = 0.15: H0 through the point path
  (the edge list holds about 4.5 million edges; nothing of size n^2 is made)
  against the oracle's Kruskal deaths computed from the same edges.
"""
import math
import os

import numpy as np
import pytest

from paper_1908_02518_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden")
U64MAX = int(np.iinfo(np.uint64).max)


def _key(bars):
    return sorted((int(b["dim"]), float(b["birth"]), float(b["death"]), int(b["birth_simplex"]),
                   U64MAX if int(b["death_simplex"]) < 0 else int(b["death_simplex"])) for b in bars)


def _coo(d, t):
    n = d.shape[0]
    i, j = np.tril_indices(n, -1)
    keep = d[i, j] <= t if math.isfinite(t) else np.ones(len(i), dtype=bool)
    return i[keep].astype(np.int32), j[keep].astype(np.int32), d[i, j][keep].astype(np.float32)


def test_clifford_torus_matches_golden():
    import torch
    import importlib.util
    import paper_1908_02518_gb300 as rg
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(GOLD, "make_golden.py"))
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    head, bars = mg.read(os.path.join(GOLD, "clifford1500.bars.txt.gz"))
    w = W.WORKLOADS["clifford1500"]()
    assert W.matrix_digest(w.dist) == head["sha256"]
    res = rg.barcodes_sparse_points(torch.from_numpy(w.points).cuda(), w.threshold, w.dim_max, w.p)
    want = sorted((d, b, e, bs, U64MAX if ds < 0 else ds) for d, b, e, bs, ds in bars)
    assert _key(res.bars) == want
    for d in range(w.dim_max + 1):
        assert res.stats[0][d]["simplices"] == head["stats"][d]["simplices"]


@pytest.mark.parametrize("case", ["torus", "ties", "z3", "cube_full"])
def test_coo_matches_oracle(oracle_mod, case):
    import paper_1908_02518_gb300 as rg
    if case == "torus":
        d, t, dm, p = W.distance_matrix(W.torus_points(300, 81)), 0.9, 2, 2
    elif case == "ties":
        d, t, dm, p = W.random_integer_matrix(30, 82, levels=4), 3.0, 2, 2
    elif case == "z3":
        d, t, dm, p = W.distance_matrix(W.sphere_points(60, 83)), 1.3, 3, 3
    else:
        d, t, dm, p = W.distance_matrix(W.cube_points(40, 84)), math.inf, 2, 2
    i, j, l = _coo(d, t)
    got = rg.barcodes_sparse(i, j, l, d.shape[0], dm, t, p)
    # missing entries are infinitely far: with every pair listed and no
    # threshold, the oracle's reference is the full complex (threshold FLT_MAX)
    want = oracle_mod.barcodes(d, dm, t if math.isfinite(t) else float(np.finfo(np.float32).max), p)
    assert _key(got.bars) == _key(want.bars)


def test_sparse_equals_dense_path():
    import torch
    import paper_1908_02518_gb300 as rg
    pts = W.torus_points(800, 85)
    d = W.distance_matrix(pts)
    dense = rg.barcodes(torch.from_numpy(d).cuda(), 2, 0.8, 2)
    sparse = rg.barcodes_sparse_points(torch.from_numpy(pts).cuda(), 0.8, 2, 2)
    assert _key(sparse.bars) == _key(dense.bars)
    for k in range(3):
        for f in ("simplices", "pairs", "essential", "apparent_cofacet", "apparent_facet", "cleared"):
            assert sparse.stats[0][k][f] == dense.stats[0][k][f], (k, f)


def test_sparse_rejects_bad_entries():
    import paper_1908_02518_gb300 as rg
    from paper_1908_02518_gb300 import _lib
    with pytest.raises(_lib.RipsError):
        rg.barcodes_sparse([0, 1], [1, 1], [0.5, 0.2], 3, 1)        # i == j
    with pytest.raises(_lib.RipsError):
        rg.barcodes_sparse([0], [5], [0.5], 3, 1)                   # vertex out of range
    with pytest.raises(_lib.RipsError):
        rg.barcodes_sparse([0], [1], [float("nan")], 3, 1)          # NaN length


def test_torus4_size_h0():
    """50,000 points on the Clifford torus at t = 0.15 (the paper's torus4
    configuration), H0, through the point path: the deaths are the lengths of a
    minimum spanning forest of the edges within t (a multiset every spanning
    forest shares), checked against scipy's minimum spanning tree of the same
    FP32 edge lengths, computed here by the documented rule from the same
    coordinates; the essential classes are the connected components."""
    import torch
    import paper_1908_02518_gb300 as rg
    scipy_spatial = pytest.importorskip("scipy.spatial")
    csgraph = pytest.importorskip("scipy.sparse.csgraph")
    import scipy.sparse as sps
    w = W.clifford(50000, 0.15, 0)
    res = rg.barcodes_sparse_points(torch.from_numpy(w.points).cuda(), 0.15, 0, 2)
    got = np.sort(res.bars["death"][np.isfinite(res.bars["death"])])
    x = w.points.astype(np.float64)
    pairs = scipy_spatial.cKDTree(x).query_pairs(0.1501, output_type="ndarray")
    diff = x[pairs[:, 0]] - x[pairs[:, 1]]
    acc = np.zeros(len(pairs))
    for k in range(x.shape[1]):  # coordinate order, each operation rounded
        acc = acc + diff[:, k] * diff[:, k]
    d32 = np.sqrt(acc).astype(np.float32)
    keep = d32 <= np.float32(0.15)
    assert (d32[keep] > 0).all()
    g = sps.coo_matrix((d32[keep].astype(np.float64), (pairs[keep, 0], pairs[keep, 1])), shape=(w.n, w.n)).tocsr()
    mst = csgraph.minimum_spanning_tree(g)
    want = np.sort(mst.data.astype(np.float32))
    assert np.array_equal(got, want)
    ncomp, _ = csgraph.connected_components(g, directed=False)
    assert int(np.isinf(res.bars["death"]).sum()) == ncomp
