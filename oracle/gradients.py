"""Reference gradients of bar endpoints (TEST INFRASTRUCTURE, float64, numpy).

A finite bar endpoint is the diameter of a simplex, i.e. the length of one of
its edges: the longest one.  When several edges tie for the longest, the edge
with the smallest combinatorial index is taken (the youngest of the tied edges
in the refined order).  With the pairing fixed, the derivative of |x_a - x_b|
with respect to x_a is (x_a - x_b) / |x_a - x_b|.  Nothing here is shared with
the CUDA path.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def simplex_vertices(index: int, d: int) -> list[int]:
    """Vertices (decreasing) of the d-simplex with the given combinatorial index:
    repeatedly the largest v with C(v, k) <= index (the Lemma of Section 4)."""
    out = []
    hi = None
    for k in range(d + 1, 0, -1):
        v = k - 1
        # grow v while C(v+1, k) <= index
        while math.comb(v + 1, k) <= index and (hi is None or v + 1 <= hi):
            v += 1
        out.append(v)
        index -= math.comb(v, k)
        hi = v - 1
    return out


def distances64(points: np.ndarray) -> np.ndarray:
    x = np.asarray(points, dtype=np.float64)
    diff = x[:, None, :] - x[None, :, :]
    return np.sqrt((diff * diff).sum(-1))


def distances32(points: np.ndarray) -> np.ndarray:
    """The FP32 matrix of the documented rule (float64 per coordinate, rounded)."""
    x = np.asarray(points, dtype=np.float64)
    acc = np.zeros((x.shape[0], x.shape[0]))
    for c in range(x.shape[1]):
        dd = x[:, None, c] - x[None, :, c]
        acc = acc + dd * dd
    return np.sqrt(acc).astype(np.float32)


def critical_edge(d32: np.ndarray, index: int, dim: int) -> tuple[int, int]:
    """Longest edge (a > b) of the simplex, ties -> smallest edge index, compared on
    the FP32 matrix the barcode was computed from."""
    v = simplex_vertices(index, dim)
    best = None
    for a, b in itertools.combinations(v, 2):  # a > b since v is decreasing
        key = (float(d32[a, b]), -(a * (a - 1) // 2 + b))
        if best is None or key > best[0]:
            best = (key, (a, b))
    return best[1]


def endpoint_edges(d32, bars):
    """(birth edge or None, death edge or None) per bar."""
    out = []
    for b in bars:
        dim = int(b["dim"])
        be = critical_edge(d32, int(b["birth_simplex"]), dim) if dim >= 1 else None
        ds = int(b["death_simplex"])
        de = critical_edge(d32, ds, dim + 1) if ds >= 0 and np.isfinite(b["death"]) else None
        out.append((be, de))
    return out


def bar_gradient(points, bars, grad_birth, grad_death) -> np.ndarray:
    """dL/dpoints (float64) given dL/dbirth and dL/ddeath per bar."""
    x = np.asarray(points, dtype=np.float64)
    d32 = distances32(points)
    g = np.zeros_like(x)
    for (be, de), gb, gd in zip(endpoint_edges(d32, bars), grad_birth, grad_death):
        for e, w in ((be, gb), (de, gd)):
            if e is None or w == 0:
                continue
            a, b = e
            diff = x[a] - x[b]
            r = math.sqrt(float(diff @ diff))
            if r > 0:
                g[a] += w * diff / r
                g[b] -= w * diff / r
    return g


def h1_loss(points64, pairs) -> float:
    """sum over H1 bars of (death - birth)^2 with fixed critical edges, float64."""
    x = np.asarray(points64, dtype=np.float64)
    s = 0.0
    for be, de in pairs:
        if be is None or de is None:
            continue
        b = math.sqrt(float(((x[be[0]] - x[be[1]]) ** 2).sum()))
        d = math.sqrt(float(((x[de[0]] - x[de[1]]) ** 2).sum()))
        s += (d - b) ** 2
    return s
