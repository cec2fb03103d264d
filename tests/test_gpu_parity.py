"""Parity of the CUDA path with the CPU oracle, bar by bar: dimension, birth,
death and the birth/death simplex indices must all be identical (the barcode
values are copies of FP32 input entries and the pairing of the refined
filtration is unique, so the comparison is exact)."""
import math

import numpy as np
import pytest

from paper_1908_02518_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U64MAX = np.iinfo(np.uint64).max


def _gpu(dist, dim_max, threshold=math.inf, p=2, device=True):
    import torch
    import paper_1908_02518_gb300 as rg
    if device:
        return rg.barcodes(torch.from_numpy(np.ascontiguousarray(dist)).cuda(), dim_max, threshold, p)
    return rg.barcodes(dist, dim_max, threshold, p)


def _key_gpu(bars):
    return sorted((int(b["dim"]), float(b["birth"]), float(b["death"]), int(b["birth_simplex"]),
                   int(b["death_simplex"])) for b in bars)


def _key_oracle(bars):
    return sorted((int(b["dim"]), float(b["birth"]), float(b["death"]), int(b["birth_simplex"]),
                   int(U64MAX) if b["death_simplex"] < 0 else int(b["death_simplex"])) for b in bars)


def assert_same(dist, dim_max, threshold=math.inf, p=2, oracle_mod=None, device=True):
    got = _gpu(dist, dim_max, threshold, p, device)
    want = oracle_mod.barcodes(dist, dim_max, threshold, p, method="coh")
    assert got.threshold == want.threshold
    g, w = _key_gpu(got.bars), _key_oracle(want.bars)
    if g != w:
        gs, ws = set(g), set(w)
        raise AssertionError(f"{len(g)} vs {len(w)} bars; only gpu: {sorted(gs - ws)[:8]}; "
                             f"only oracle: {sorted(ws - gs)[:8]}")
    # statistics against the oracle's counts (apparent pairs are pairs too)
    for d in range(dim_max + 1):
        s, o = got.stats[0][d], want.stats[d]
        assert s["simplices"] == o["simplices"], d
        assert s["essential"] == o["essential"], d
        if d >= 1:
            assert s["simplices"] == s["apparent_cofacet"] + s["apparent_facet"] + s["cleared"] + s["columns"]
            assert s["pairs"] + s["apparent_cofacet"] == o["pairs"], d
    return got


def test_rectangle(oracle_mod):
    d = W.distance_matrix(W.rectangle())
    got = assert_same(d, 2, oracle_mod=oracle_mod)
    assert [(int(b["dim"]), float(b["birth"]), float(b["death"])) for b in got.dim(1)] == [(1, 4.0, 5.0)]


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_tiny(oracle_mod, n):
    d = W.distance_matrix(W.cube_points(n, 10 + n))
    assert_same(d, 2, oracle_mod=oracle_mod)


@pytest.mark.parametrize("seed", range(6))
def test_random_clouds(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(8, 40))
    d = W.distance_matrix(rng.random((n, 3)).astype(np.float32))
    dm = [1, 2, 3][seed % 3] if n <= 24 else 2
    p = [2, 3, 5][seed % 3]
    th = math.inf if seed % 2 == 0 else float(np.quantile(d[d > 0], 0.4))
    assert_same(d, dm, th, p, oracle_mod=oracle_mod)


@pytest.mark.parametrize("seed", range(4))
def test_ties(oracle_mod, seed):
    """Integer distances: many equal diameters, so the index tie-break decides."""
    n = 14 + 3 * seed
    d = W.random_integer_matrix(n, 200 + seed, 4)
    assert_same(d, 2, math.inf, [2, 3][seed % 2], oracle_mod=oracle_mod)


@pytest.mark.parametrize("n", [5, 6, 9, 12])
def test_regular_polygon(oracle_mod, n):
    assert_same(W.regular_polygon_matrix(n), 1, oracle_mod=oracle_mod)


def test_octahedron(oracle_mod):
    for p in (2, 3):
        assert_same(W.octahedron_matrix(), 2, p=p, oracle_mod=oracle_mod)


def test_host_path_equals_device_path(oracle_mod):
    d = W.distance_matrix(W.torus_points(60, 3))
    a = _gpu(d, 2, 1.2, 2, device=True)
    b = _gpu(d, 2, 1.2, 2, device=False)
    assert np.array_equal(a.bars, b.bars)


def test_cube100(oracle_mod):
    w = W.cube_100()
    assert_same(w.dist, w.dim_max, w.threshold, w.p, oracle_mod=oracle_mod)


def test_torus1000(oracle_mod):
    w = W.torus_1000()
    assert_same(w.dist, w.dim_max, w.threshold, w.p, oracle_mod=oracle_mod)


def test_sphere_s3_small_z3(oracle_mod):
    """Dimension 3 over Z/3 on a smaller sample of the S^3 workload."""
    d = W.distance_matrix(W.sphere_points(48, 1005, 4))
    assert_same(d, 3, math.inf, 3, oracle_mod=oracle_mod)


def test_bad_input_status():
    import paper_1908_02518_gb300 as rg
    d = W.distance_matrix(W.cube_points(10, 1))
    d[5, 2] = np.nan
    with pytest.raises(rg.RipsError) as e:
        _gpu(d, 1)
    assert e.value.status == -1
    d[5, 2] = -0.5
    with pytest.raises(rg.RipsError):
        _gpu(d, 1)


def test_batched_equals_single(oracle_mod):
    import torch
    import paper_1908_02518_gb300 as rg
    clouds = [W.cube_points(n, 300 + n) for n in (12, 30, 7, 45)]
    off = np.concatenate([[0], np.cumsum([c.shape[0] for c in clouds])])
    x = torch.from_numpy(np.concatenate(clouds)).cuda()
    res = rg.barcodes_batched(x, off, dim_max=1)
    for c, pts in enumerate(clouds):
        want = oracle_mod.barcodes(W.distance_matrix(pts), 1)
        assert _key_gpu(res.dim(0, c)) + _key_gpu(res.dim(1, c)) == _key_oracle(want.bars)


def test_device_distance_rule_matches_host():
    import torch
    import paper_1908_02518_gb300 as rg
    pts = W.so3_points(300, 5)
    d_host = W.distance_matrix(pts)
    d_dev = rg.distance_matrix(torch.from_numpy(pts).cuda()).cpu().numpy()
    assert np.array_equal(d_host, d_dev)
