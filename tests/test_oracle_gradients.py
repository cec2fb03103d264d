"""Pins for oracle/gradients.py, the CPU reference of the backward pass.

Each check is independent of the code it tests:
  * simplex_vertices against the values the paper prints for the combinatorial
    number system (Section 2) and against brute force over every k-subset;
  * critical_edge against the barcode: the FP32 length of the edge it names is
    the bar's birth or death value, which the C oracle's reduction produced;
  * the tie rule (a reading the paper leaves open: among equal longest edges the
    one with the smallest colex index, i.e. the edge that enters the refined
    filtration last and so admits the simplex) against the oracle's own
    filtration order, on matrices with many ties, and on two hand-built ties;
  * bar_gradient for loss = sum over H1 bars of (death - birth)^2 against
    float64 central finite differences (step 1e-4) of the same loss, where the
    loss is evaluated at each perturbed point set from the oracle's pairs there
    and the float64 diameters of those simplices (decoded by the C oracle, not
    by gradients.py); coordinates whose pairing changes within +-h are skipped.
    Tolerance: ||g - g_fd||_inf <= 1e-4 max(||g_fd||_inf, 1e-6).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import gradients as G
from paper_1908_02518_gb300 import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
STEP = 1e-4
TOL = 1e-4


def test_simplex_vertices_paper_values():
    with open(os.path.join(GOLD, "combinatorial_number_system.json")) as f:
        g = json.load(f)
    for verts, idx in g["table_d2"] + [g["example"]]:
        assert G.simplex_vertices(idx, 2) == verts
    for verts, idx in g["cofacets_of_530_n7"]:
        assert G.simplex_vertices(idx, 3) == verts


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_simplex_vertices_brute_force(k):
    """Every k-subset of {0..11}: index = sum_l C(a_l, l + 1) over increasing
    vertices a_0 < ... (Section 2) decodes back to the subset."""
    for sub in itertools.combinations(range(12), k):
        idx = sum(math.comb(a, l + 1) for l, a in enumerate(sub))
        assert G.simplex_vertices(idx, k - 1) == sorted(sub, reverse=True)


def _edge_index(a, b):
    return a * (a - 1) // 2 + b  # a > b


def _clouds():
    rng = np.random.Generator(np.random.PCG64(9100))
    return [W.circle_points(rng, 36, 0.05).astype(np.float32),
            W._torus(rng, 36, 2.0, 1.0, 0.02).astype(np.float32),
            rng.random((34, 3)).astype(np.float32)]


def test_critical_edge_length_is_bar_value(oracle_mod):
    for pts in _clouds():
        d32 = G.distances32(pts)
        r = oracle_mod.barcodes(d32, 2)
        fin = 0
        for b in r.bars:
            dim = int(b["dim"])
            if dim >= 1:
                a, c = G.critical_edge(d32, int(b["birth_simplex"]), dim)
                assert d32[a, c] == b["birth"]
            if np.isfinite(b["death"]):
                a, c = G.critical_edge(d32, int(b["death_simplex"]), dim + 1)
                assert d32[a, c] == b["death"]
                fin += 1
        assert fin > 10


def test_critical_edge_hand_built_ties():
    # edges of the triangle {0, 1, 2}: (1,0) index 0, (2,0) index 1, (2,1) index 2
    d = np.zeros((3, 3), dtype=np.float32)
    d[1, 0] = d[0, 1] = 1.0
    d[2, 0] = d[0, 2] = 2.0
    d[2, 1] = d[1, 2] = 2.0
    assert G.critical_edge(d, 0, 2) == (2, 0)   # ties 1 and 2: index 1 wins
    d[1, 0] = d[0, 1] = 2.0
    d[2, 0] = d[0, 2] = 1.0
    assert G.critical_edge(d, 0, 2) == (1, 0)   # ties 0 and 2: index 0 wins


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_critical_edge_is_youngest_edge_in_filtration(oracle_mod, seed):
    """On integer distances (many ties) the critical edge of every simplex of
    dimension 1..3 is the edge that comes last in the oracle's refined order."""
    d = W.random_integer_matrix(9, seed, levels=3)
    dims, idx, _ = oracle_mod.filtration(d, 3)
    pos = {(int(k), int(i)): q for q, (k, i) in enumerate(zip(dims, idx))}
    for (k, i) in pos:
        if k < 1:
            continue
        v = G.simplex_vertices(i, k)
        youngest = max(itertools.combinations(v, 2), key=lambda e: pos[(1, _edge_index(*e))])
        assert G.critical_edge(d, i, k) == youngest


def _h1_pairs(oracle_mod, x64):
    d32 = G.distances32(x64)
    bars = oracle_mod.barcodes(d32, 1).dim(1)
    bars = bars[np.isfinite(bars["death"])]
    return bars, tuple(sorted((int(b["birth_simplex"]), int(b["death_simplex"])) for b in bars))


def _diam64(oracle_mod, x64, idx, dim, n):
    v = oracle_mod.simplex_vertices(idx, dim, n)
    return max(math.sqrt(float(((x64[a] - x64[b]) ** 2).sum())) for a, b in itertools.combinations(v, 2))


def _loss(oracle_mod, x64, key):
    n = x64.shape[0]
    return sum((_diam64(oracle_mod, x64, de, 2, n) - _diam64(oracle_mod, x64, bi, 1, n)) ** 2 for bi, de in key)


@pytest.mark.parametrize("which", [0, 1, 2])
def test_bar_gradient_matches_finite_differences(oracle_mod, which):
    pts = _clouds()[which]
    x0 = pts.astype(np.float64)
    bars, key = _h1_pairs(oracle_mod, x0)
    assert len(bars) >= 1
    diff = bars["death"].astype(np.float64) - bars["birth"].astype(np.float64)
    g = G.bar_gradient(pts, bars, -2 * diff, 2 * diff)
    fd = np.full(x0.shape, np.nan)
    skipped = 0
    for i in range(x0.shape[0]):
        for c in range(x0.shape[1]):
            vals = []
            for s in (+1, -1):
                x = x0.copy()
                x[i, c] += s * STEP
                _, k2 = _h1_pairs(oracle_mod, x)
                if k2 != key:
                    break
                vals.append(_loss(oracle_mod, x, key))
            if len(vals) < 2:
                skipped += 1
                continue
            fd[i, c] = (vals[0] - vals[1]) / (2 * STEP)
    m = ~np.isnan(fd)
    assert skipped <= x0.size // 10, skipped
    scale = max(np.abs(fd[m]).max(), 1e-6)
    err = np.abs(g[m] - fd[m]).max()
    assert err <= TOL * scale, (err, scale, skipped)
    assert np.abs(fd[m]).max() > 0  # the loss moves: the check is not vacuous
