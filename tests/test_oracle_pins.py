"""Pins for the CPU oracle: values the paper prints, closed forms, invariants
and brute force.  These run without a GPU."""
import itertools
import json
import math
import os

import numpy as np
import pytest

from brute_rank import brute_barcode
from conftest import bars_as_tuples
from paper_1908_02518_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
FMAX = float(np.finfo(np.float32).max)  # a threshold that admits every simplex


def gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


# ---------------------------------------------------------------- worked example

def test_rectangle_distance_matrix():
    g = gold("rectangle.json")
    d = W.distance_matrix(np.array(g["points"], dtype=np.float32))
    assert np.array_equal(d, np.array(g["distance_matrix"], dtype=np.float32))


@pytest.mark.parametrize("method", ["def", "coh"])
def test_rectangle_filtration_order(oracle_mod, method):
    """Section 2: the simplices of the rectangle in refined filtration order."""
    g = gold("rectangle.json")
    d = np.array(g["distance_matrix"], dtype=np.float32)
    dims, idx, diam = oracle_mod.filtration(d, 3)
    got = [oracle_mod.simplex_vertices(int(i), int(k), 4) for k, i in zip(dims, idx)]
    assert got == g["filtration_simplices"]
    assert diam.tolist() == g["filtration_diameters"]


def test_rectangle_boundary_matrices(oracle_mod):
    """Section 3.5: the filtration boundary matrices d1, d2, d3 (over Z/2)."""
    g = gold("rectangle.json")
    d = np.array(g["distance_matrix"], dtype=np.float32)
    full = oracle_mod.boundary_matrix(d, 3, p=2)
    order = [tuple(s) for s in g["filtration_simplices"]]
    pos = {s: i for i, s in enumerate(order)}
    for key in ("boundary_1", "boundary_2", "boundary_3"):
        blk = g[key]
        rows = [pos[tuple(r)] for r in blk["rows"]]
        cols = [pos[tuple(c)] for c in blk["columns"]]
        assert full[np.ix_(rows, cols)].tolist() == blk["matrix"], key


def test_rectangle_boundary_signs_z3(oracle_mod):
    """Over Z/3 the columns are oriented boundaries: d o d = 0."""
    g = gold("rectangle.json")
    d = np.array(g["distance_matrix"], dtype=np.float32)
    m = oracle_mod.boundary_matrix(d, 3, p=3)
    assert not ((m @ m) % 3).any()
    assert set(np.unique(m)) <= {0, 1, 2}


def test_rectangle_apparent_pairs(oracle_mod):
    """Section 3.5: the five apparent pairs of the rectangle."""
    g = gold("rectangle.json")
    d = np.array(g["distance_matrix"], dtype=np.float32)
    order = g["filtration_simplices"]
    pairs = oracle_mod.apparent_pairs(d, 3)
    got = sorted([order[s], order[t]] for s, t in pairs)
    assert got == sorted(g["apparent_pairs"])


def test_rectangle_discrete_morse_function(oracle_mod):
    """Section 3.5: f(sigma_j) = i for an apparent pair (sigma_i, sigma_j), else j."""
    g = gold("rectangle.json")
    d = np.array(g["distance_matrix"], dtype=np.float32)
    pairs = oracle_mod.apparent_pairs(d, 3)
    f = list(range(15))
    for s, t in pairs:
        f[t] = s
    assert f == g["morse_function"]


@pytest.mark.parametrize("method", ["def", "coh"])
def test_rectangle_barcode(oracle_mod, method):
    g = gold("rectangle.json")
    d = np.array(g["distance_matrix"], dtype=np.float32)
    r = oracle_mod.barcodes(d, 2, method=method)
    want = [(0, float(b), float(e)) for b, e in g["barcode_H0"]] + \
           [(1, float(b), float(e)) for b, e in g["barcode_H1"]]
    assert bars_as_tuples(r.bars) == sorted(want)
    # the H1 bar is born by the edge (2,0) and killed by the triangle (3,1,0)
    h1 = r.dim(1)[0]
    assert oracle_mod.simplex_vertices(int(h1["birth_simplex"]), 1, 4) == [2, 0]
    assert oracle_mod.simplex_vertices(int(h1["death_simplex"]), 2, 4) == [3, 1, 0]


# ---------------------------------------------------- combinatorial number system

def test_number_system_values(oracle_mod):
    g = gold("combinatorial_number_system.json")
    for verts, want in g["table_d2"]:
        assert oracle_mod.simplex_index(verts) == want
    verts, want = g["example"]
    assert oracle_mod.simplex_index(verts) == want
    for verts, want in g["cofacets_of_530_n7"]:
        assert oracle_mod.simplex_index(verts) == want
    n = 9
    assert oracle_mod.simplex_index([n - 1, n - 2, n - 3]) == math.comb(n, 3) - 1


def test_number_system_round_trip(oracle_mod):
    """Index = rank in colexicographic order, and decoding inverts it."""
    for n in range(1, 15):
        for d in range(0, min(n, 5)):
            combos = sorted(itertools.combinations(range(n), d + 1), key=lambda c: c[::-1])
            for rank, c in enumerate(combos):
                desc = list(c[::-1])
                assert oracle_mod.simplex_index(desc) == rank
                if n <= 10 or rank % 17 == 0:
                    assert oracle_mod.simplex_vertices(rank, d, n) == desc


# ------------------------------------------------------------------ brute force

def _random_cases():
    rng = np.random.default_rng(12345)
    cases = []
    for trial in range(36):
        n = int(rng.integers(2, 8))
        dm = int(rng.integers(0, 3))
        p = (2, 3, 5)[trial % 3]
        if trial % 2:
            d = W.random_integer_matrix(n, trial, 3 + trial % 3)
        else:
            d = W.distance_matrix(rng.random((n, 3)).astype(np.float32))
        th = math.inf if trial % 4 != 3 else float(np.median(d[d > 0]))
        cases.append((d, dm, th, p))
    return cases


@pytest.mark.parametrize("method", ["def", "coh"])
def test_brute_force_rank_invariant(oracle_mod, method):
    """Barcode = interval decomposition of the rank invariant (tiny inputs)."""
    for d, dm, th, p in _random_cases():
        got = bars_as_tuples(oracle_mod.barcodes(d, dm, th, p, method=method).bars)
        assert got == brute_barcode(d, dm, th, p), (d, dm, th, p)


def test_brute_force_dim3(oracle_mod):
    rng = np.random.default_rng(7)
    for seed in range(4):
        d = W.distance_matrix(rng.random((7, 4)).astype(np.float32))
        for p in (2, 3):
            got = bars_as_tuples(oracle_mod.barcodes(d, 3, p=p, method="coh").bars)
            assert got == brute_barcode(d, 3, math.inf, p)


def test_homology_equals_cohomology_pairs(oracle_mod):
    """Both methods give the same persistence pairs, simplex by simplex,
    including the zero-persistence ones (the pairing is unique)."""
    rng = np.random.default_rng(99)
    for trial in range(12):
        n = int(rng.integers(6, 16))
        dm = int(rng.integers(1, 3))
        p = (2, 3)[trial % 2]
        d = (W.random_integer_matrix(n, 100 + trial, 6) if trial % 3 == 0
             else W.distance_matrix(rng.random((n, 3)).astype(np.float32)))
        a = oracle_mod.barcodes(d, dm, p=p, method="def", keep_zero=True)
        b = oracle_mod.barcodes(d, dm, p=p, method="coh", keep_zero=True)
        assert np.array_equal(a.bars, b.bars)
        for k in range(dm + 1):
            for f in ("simplices", "pairs", "zero_pairs", "essential"):
                assert a.stats[k][f] == b.stats[k][f]


# ------------------------------------------------------------------ H0 / Kruskal

def _prim_mst_lengths(d):
    n = d.shape[0]
    full = np.tril(d, -1).astype(np.float64)
    full = full + full.T
    inside = np.zeros(n, bool)
    inside[0] = True
    best = full[0].copy()
    out = []
    for _ in range(n - 1):
        best[inside] = np.inf
        j = int(np.argmin(best))
        out.append(float(np.float32(best[j])))
        inside[j] = True
        best = np.minimum(best, full[j])
    return sorted(out)


@pytest.mark.parametrize("method", ["def", "coh"])
def test_h0_deaths_are_mst_lengths(oracle_mod, method):
    rng = np.random.default_rng(3)
    for n in (5, 17, 40):
        d = W.distance_matrix(rng.random((n, 3)).astype(np.float32))
        r = oracle_mod.barcodes(d, 0, threshold=FMAX, method=method, keep_zero=True)
        h0 = r.dim(0)
        finite = sorted(float(x) for x in h0["death"] if np.isfinite(x))
        assert finite == _prim_mst_lengths(d)
        assert np.isinf(h0["death"]).sum() == 1


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("n", list(range(4, 13)))
def test_regular_polygon_single_h1_bar(oracle_mod, n):
    """Regular n-gon: one H1 bar [chord(1), chord(ceil(n/3))) (cyclic Rips)."""
    d = W.regular_polygon_matrix(n)
    r = oracle_mod.barcodes(d, 1, p=3)
    h1 = r.dim(1)
    assert len(h1) == 1
    assert float(h1["birth"][0]) == float(d[0, 1])
    assert float(h1["death"][0]) == float(d[0, -(-n // 3)])


def test_octahedron(oracle_mod):
    d = W.octahedron_matrix()
    for method in ("def", "coh"):
        for p in (2, 3):
            r = oracle_mod.barcodes(d, 2, p=p, method=method)
            s2 = float(np.float32(math.sqrt(2)))
            want = [(0, 0.0, s2)] * 5 + [(0, 0.0, math.inf), (2, s2, 2.0)]
            assert bars_as_tuples(r.bars) == sorted(want)


@pytest.mark.parametrize("n", [2, 3, 5, 8])
def test_regular_simplex(oracle_mod, n):
    d = W.regular_simplex_matrix(n)
    for method in ("def", "coh"):
        r = oracle_mod.barcodes(d, min(3, n - 1), method=method)
        assert bars_as_tuples(r.bars) == sorted([(0, 0.0, 1.0)] * (n - 1) + [(0, 0.0, math.inf)])


def test_single_point(oracle_mod):
    d = np.zeros((1, 1), dtype=np.float32)
    for method in ("def", "coh"):
        r = oracle_mod.barcodes(d, 2, method=method)
        assert bars_as_tuples(r.bars) == [(0, 0.0, math.inf)]


# ------------------------------------------------------------------ counts

@pytest.mark.parametrize("method", ["def", "coh"])
def test_pair_count_identity(oracle_mod, method):
    """Every d-simplex is a birth (paired or essential) or kills a (d-1)-class."""
    rng = np.random.default_rng(5)
    for n, dm, th in ((20, 2, math.inf), (30, 1, 0.5), (12, 3, math.inf)):
        d = W.distance_matrix(rng.random((n, 3)).astype(np.float32))
        r = oracle_mod.barcodes(d, dm, th, method=method)
        for k in range(dm + 1):
            s = r.stats[k]
            below = r.stats[k - 1]["pairs"] if k else 0
            assert s["simplices"] == below + s["pairs"] + s["essential"]
            assert s["simplices"] == oracle_mod.count_simplices(d, k, th)


def test_full_complex_pair_counts(oracle_mod):
    """Full complex: #pairs(d) = C(n, d+1) - #pairs(d-1), no essentials above H0."""
    d = W.distance_matrix(W.cube_points(25, 8))
    r = oracle_mod.barcodes(d, 2, threshold=FMAX)
    prev = 0
    for k in range(3):
        assert r.stats[k]["pairs"] == math.comb(25, k + 1) - prev - (1 if k == 0 else 0)
        prev = r.stats[k]["pairs"]


def test_paper_column_counts_n192(oracle_mod):
    """Section 3.3: cohomology with clearing on the 3-skeleton of the full simplex
    on 192 vertices reduces 1,161,472 columns; Table 2 (sphere3): 18,145 and
    1,143,135 pairs in dimensions 1 and 2."""
    g = gold("column_counts.json")
    d = W.distance_matrix(W.sphere_points(g["n"], 77, 3))
    r = oracle_mod.barcodes(d, g["max_degree"], threshold=FMAX, method="coh")
    assert sum(s["columns"] for s in r.stats) == g["cohomology_clearing_columns"]
    assert sum(s["pairs"] for s in r.stats) == g["death_columns"]
    assert r.stats[1]["pairs"] == g["total_pairs_dim1"]
    assert r.stats[2]["pairs"] == g["total_pairs_dim2"]


# ------------------------------------------------------------------ apparent pairs

def test_apparent_pairs_are_persistence_pairs(oracle_mod):
    """Lemma (Section 3.5): every apparent pair is a persistence pair, and no
    simplex is in two apparent pairs."""
    rng = np.random.default_rng(11)
    for trial in range(6):
        n = 9 if trial < 3 else 7
        d = (W.random_integer_matrix(n, 50 + trial, 4) if trial % 2
             else W.distance_matrix(rng.random((n, 3)).astype(np.float32)))
        dims, idx, diam = oracle_mod.filtration(d, 3)
        pairs = oracle_mod.apparent_pairs(d, 3)
        r = oracle_mod.barcodes(d, 2, method="def", keep_zero=True)
        pp = {(int(b["dim"]), int(b["birth_simplex"]), int(b["death_simplex"])) for b in r.bars}
        used = set()
        for s, t in pairs:
            assert s not in used and t not in used
            used |= {s, t}
            if dims[s] <= 2:
                assert (int(dims[s]), int(idx[s]), int(idx[t])) in pp


def test_dim1_zero_pairs_are_apparent(oracle_mod):
    """Theorem (Section 3.5): with distinct distances, the zero-persistence pairs
    in dimension 1 are exactly the apparent pairs."""
    rng = np.random.default_rng(21)
    for _ in range(4):
        d = W.distance_matrix(rng.random((10, 3)).astype(np.float32))
        r = oracle_mod.barcodes(d, 1, threshold=FMAX, method="def", keep_zero=True)
        zero = {(int(b["birth_simplex"]), int(b["death_simplex"]))
                for b in r.dim(1) if b["birth"] == b["death"]}
        dims, idx, diam = oracle_mod.filtration(d, 2, threshold=FMAX)
        app = {(int(idx[s]), int(idx[t])) for s, t in oracle_mod.apparent_pairs(d, 2, threshold=FMAX)
               if dims[s] == 1 and diam[s] == diam[t]}
        assert zero == app
        assert r.stats[1]["apparent_zero"] == len(app)


# ------------------------------------------------------------------ threshold

def test_enclosing_radius_gives_full_barcode(oracle_mod):
    """Section 4 'Input': above the enclosing radius the complex is a cone, so
    thresholding there changes no bar."""
    rng = np.random.default_rng(4)
    for n in (8, 15, 30):
        d = W.distance_matrix(rng.random((n, 3)).astype(np.float32))
        a = oracle_mod.barcodes(d, 2 if n < 30 else 1)
        b = oracle_mod.barcodes(d, 2 if n < 30 else 1, threshold=FMAX)
        assert np.array_equal(a.bars, b.bars)
        assert a.threshold == oracle_mod.enclosing_radius(d)


def test_threshold_is_inclusive(oracle_mod):
    d = np.array([[0, 1], [1, 0]], dtype=np.float32)
    assert bars_as_tuples(oracle_mod.barcodes(d, 0, 1.0).bars) == [(0, 0.0, 1.0), (0, 0.0, math.inf)]
    assert bars_as_tuples(oracle_mod.barcodes(d, 0, 0.999).bars) == [(0, 0.0, math.inf)] * 2


def test_bad_arguments(oracle_mod):
    d = W.distance_matrix(W.cube_points(5, 1))
    for kw in ({"p": 4}, {"p": 1}, {"p": 65537}):
        with pytest.raises(oracle_mod.OracleError):
            oracle_mod.barcodes(d, 1, **kw)
    bad = d.copy()
    bad[3, 1] = -1.0
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.barcodes(bad, 1)
    bad[3, 1] = np.nan
    with pytest.raises(oracle_mod.OracleError):
        oracle_mod.barcodes(bad, 1)
