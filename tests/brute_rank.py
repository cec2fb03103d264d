"""Brute-force barcode from the rank invariant (independent of any reduction).

For tiny inputs the barcode is recomputed straight from its definition as the
interval decomposition of the persistence module H_d(K_s) -> H_d(K_t): for every
pair of filtration values s <= t,

    rank(H_d(K_s) -> H_d(K_t)) = dim Z_d(K_s) - dim(B_d(K_t) restricted to K_s),

with dim Z_d(K_s) = #d-simplices(s) - rank boundary_d(s) and the second term
= rank boundary_{d+1}(t) - rank(rows of boundary_{d+1}(t) outside K_s).  Bar
multiplicities follow by inclusion-exclusion over consecutive values.  All
ranks are taken over Z/p by Gaussian elimination.  Nothing here is shared with
the oracle or with the CUDA path.
"""
from __future__ import annotations

import itertools
import math

import numpy as np


def rank_mod_p(m: np.ndarray, p: int) -> int:
    a = np.array(m, dtype=np.int64) % p
    if a.size == 0:
        return 0
    rows, cols = a.shape
    r = 0
    for c in range(cols):
        piv = None
        for i in range(r, rows):
            if a[i, c] % p:
                piv = i
                break
        if piv is None:
            continue
        a[[r, piv]] = a[[piv, r]]
        inv = pow(int(a[r, c]), p - 2, p)
        a[r] = (a[r] * inv) % p
        for i in range(rows):
            if i != r and a[i, c]:
                a[i] = (a[i] - a[i, c] * a[r]) % p
        r += 1
        if r == rows:
            break
    return r


def enclosing_radius(d: np.ndarray) -> np.float32:
    n = d.shape[0]
    if n == 1:
        return np.float32(0)
    full = np.tril(d, -1)
    full = full + full.T
    return np.float32(min(max(full[i, j] for j in range(n) if j != i) for i in range(n)))


def brute_barcode(dist: np.ndarray, dim_max: int, threshold: float = math.inf, p: int = 2):
    """Sorted list of (dim, birth, death) with death = inf for essential bars."""
    d = np.asarray(dist, dtype=np.float32)
    n = d.shape[0]
    full = np.tril(d, -1)
    full = full + full.T
    t = enclosing_radius(d) if (math.isinf(threshold) or math.isnan(threshold)) else np.float32(threshold)

    def diam(s):
        return max((full[a, b] for a, b in itertools.combinations(s, 2)), default=np.float32(0))

    simp = {k: [] for k in range(dim_max + 2)}
    for k in range(dim_max + 2):
        for s in itertools.combinations(range(n), k + 1):
            v = diam(s)
            if v <= t:
                simp[k].append((s, v))
    values = sorted({float(v) for k in simp for _, v in simp[k]})
    m = len(values)
    bars = []
    for k in range(dim_max + 1):
        rows_k = simp[k]
        cols_up = simp[k + 1]
        pos_k = {s: i for i, (s, _) in enumerate(rows_k)}
        # boundary_{k+1}: rows k-simplices, columns (k+1)-simplices
        bd_up = np.zeros((len(rows_k), len(cols_up)), dtype=np.int64)
        for j, (s, _) in enumerate(cols_up):
            for q in range(len(s)):
                f = s[:q] + s[q + 1:]
                bd_up[pos_k[f], j] = 1 if q % 2 == 0 else p - 1
        if k > 0:
            rows_km = simp[k - 1]
            pos_km = {s: i for i, (s, _) in enumerate(rows_km)}
            bd_k = np.zeros((len(rows_km), len(rows_k)), dtype=np.int64)
            for j, (s, _) in enumerate(rows_k):
                for q in range(len(s)):
                    f = s[:q] + s[q + 1:]
                    bd_k[pos_km[f], j] = 1 if q % 2 == 0 else p - 1
        kval = np.array([float(v) for _, v in rows_k])
        uval = np.array([float(v) for _, v in cols_up])

        def rk(a, b):
            """rank H_k(K_{values[a]}) -> H_k(K_{values[b]}), a <= b, 0-based."""
            if a < 0:
                return 0
            sa, sb = values[a], values[b]
            in_a = kval <= sa
            nz = int(in_a.sum())
            zdim = nz - (rank_mod_p(bd_k[:, in_a], p) if k > 0 else 0)
            cu = uval <= sb
            mb = bd_up[:, cu]
            bdim = rank_mod_p(mb, p)
            outside = rank_mod_p(mb[~in_a, :], p)
            return zdim - (bdim - outside)

        cache = {}

        def r(a, b):
            if (a, b) not in cache:
                cache[(a, b)] = rk(a, b)
            return cache[(a, b)]

        for a in range(m):
            for b in range(a + 1, m):
                mult = r(a, b - 1) - r(a - 1, b - 1) - r(a, b) + r(a - 1, b)
                bars += [(k, values[a], values[b])] * mult
            mult = r(a, m - 1) - r(a - 1, m - 1)
            bars += [(k, values[a], math.inf)] * mult
    return sorted(bars)
