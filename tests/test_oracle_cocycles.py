"""Representative cocycles of the oracle (Sections 3.1 and 3.4: R = D V, and the
column V_j of a bar's birth simplex represents its class), pinned by brute force
on small complexes independent of the oracle: coboundaries from the definition,
cohomology classes by ranks over Z/p, and the pairing of an H1 cocycle with the
cycle of a polygon."""
import itertools
import math

import numpy as np
import pytest

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def _oracle():
    import oracle
    return oracle


def _index(verts):
    """combinatorial number system: sum over the ascending vertices of C(a_l, l + 1)"""
    return sum(math.comb(a, l + 1) for l, a in enumerate(sorted(verts)))


def _complex(d, k, t):
    """k-simplices of the Rips complex of d at threshold t: sorted vertex tuples -> diameter"""
    n = d.shape[0]
    out = {}
    for s in itertools.combinations(range(n), k + 1):
        diam = max((float(d[a, b]) for a, b in itertools.combinations(s, 2)), default=0.0)
        if diam <= t:
            out[s] = diam
    return out


def _coboundary(z, taus, p):
    """(delta z)(tau) = sum_q (-1)^q z(tau without its q-th vertex), over Z/p"""
    out = {}
    for tau in taus:
        c = 0
        for q in range(len(tau)):
            face = tau[:q] + tau[q + 1:]
            c += (-1) ** q * z.get(_index(face), 0)
        c %= p
        if c:
            out[tau] = c
    return out


def _rank_mod_p(rows, p):
    """rank over Z/p of a list of equal-length integer rows"""
    m = [list(r) for r in rows]
    rank, col = 0, 0
    ncols = len(m[0]) if m else 0
    while rank < len(m) and col < ncols:
        piv = next((i for i in range(rank, len(m)) if m[i][col] % p), None)
        if piv is None:
            col += 1
            continue
        m[rank], m[piv] = m[piv], m[rank]
        inv = pow(m[rank][col], p - 2, p)
        m[rank] = [(x * inv) % p for x in m[rank]]
        for i in range(len(m)):
            if i != rank and m[i][col] % p:
                f = m[i][col]
                m[i] = [(a - f * b) % p for a, b in zip(m[i], m[rank])]
        rank += 1
        col += 1
    return rank


def _is_coboundary(z, lower, simplices, p):
    """is the d-cochain z (index -> coef) delta of some (d-1)-cochain on these simplices?"""
    order = sorted(simplices)
    pos = {s: i for i, s in enumerate(order)}
    # columns: delta of each (d-1)-simplex restricted to `simplices`
    cols = []
    for f in lower:
        col = [0] * len(order)
        for s in order:
            if set(f) <= set(s):
                q = next(i for i, v in enumerate(s) if v not in f)
                col[pos[s]] = (-1) ** q % p
        cols.append(col)
    zc = [z.get(_index(s), 0) % p for s in order]
    if not cols:
        return not any(zc)
    return _rank_mod_p(cols + [zc], p) == _rank_mod_p(cols, p)


def _older(a, b):
    """refined filtration order on simplices of one dimension: diameter, then larger index first"""
    return a[0] < b[0] or (a[0] == b[0] and a[1] > b[1])


def _with_bars(o, d, dim_max, p):
    """the smallest tested threshold (quantile of the edge lengths) with a bar of dimension >= 1"""
    lengths = np.sort(d[np.triu_indices(d.shape[0], 1)])
    for q in (0.3, 0.4, 0.5, 0.6, 0.7, 0.8, 0.9):
        t = float(lengths[int(q * (len(lengths) - 1))])
        res = o.barcodes(d, dim_max, t, p, cocycles=True)
        if (res.bars["dim"] >= 1).any():
            return t, res
    raise AssertionError("no bar of dimension >= 1 at any tested threshold")


def _clouds():
    """small clouds with classes in H1 and H2: a noisy circle, two noisy
    circles, a noisy 2-sphere, a slightly irregular 7-gon"""
    rng = np.random.Generator(np.random.PCG64(4242))

    def dist(x):
        return np.sqrt(((x[:, None] - x[None]) ** 2).sum(-1)).astype(np.float32)

    def circle(m, r=1.0, c=(0.0, 0.0), noise=0.05):
        th = rng.random(m) * 2 * np.pi
        return np.stack([c[0] + r * np.cos(th), c[1] + r * np.sin(th)], 1) + noise * rng.standard_normal((m, 2))

    sphere = rng.standard_normal((12, 3))
    sphere /= np.linalg.norm(sphere, axis=1, keepdims=True)
    th = np.linspace(0, 2 * np.pi, 7, endpoint=False) + 0.01 * rng.random(7)
    return [dist(circle(9)),
            dist(np.concatenate([circle(5, 0.6), circle(5, 0.6, (2.0, 0.0))])),
            dist(sphere + 0.03 * rng.standard_normal((12, 3))),
            dist(np.stack([np.cos(th), np.sin(th)], 1))]


@pytest.mark.parametrize("p", [2, 3])
@pytest.mark.parametrize("case", range(4))
def test_cocycles_reduce_to_their_pivots(case, p):
    """delta V_j is zero on every (d+1)-simplex older than the death simplex and
    not zero on it; an essential class's cocycle has no coboundary at all; V_j
    holds its birth simplex with coefficient 1 and otherwise only younger ones."""
    o = _oracle()
    d = _clouds()[case]
    t, res = _with_bars(o, d, 2, p)
    seen = 0
    for bar, (idx, cf) in zip(res.bars, res.cocycles):
        k = int(bar["dim"])
        if k == 0:
            assert len(idx) == 0
            continue
        seen += 1
        lower = _complex(d, k, t)
        upper = _complex(d, k + 1, t)
        by_index = {_index(s): s for s in lower}
        z = {int(i): int(c) for i, c in zip(idx, cf)}
        assert all(i in by_index for i in z), "cocycle entries are simplices of the complex"
        bs = int(bar["birth_simplex"])
        assert z.get(bs) == 1
        bkey = (lower[by_index[bs]], bs)
        for i in z:
            if i != bs:
                assert _older(bkey, (lower[by_index[i]], i)), "other entries are younger than the birth simplex"
        dz = _coboundary(z, list(upper), p)
        if not np.isfinite(bar["death"]):
            assert dz == {}
        else:
            ds = int(bar["death_simplex"])
            tau = next(s for s in upper if _index(s) == ds)
            assert dz.get(tau, 0) != 0
            dkey = (upper[tau], ds)
            for s, c in dz.items():
                assert not _older((upper[s], _index(s)), dkey), "no coboundary before the death simplex"
    assert seen > 0


@pytest.mark.parametrize("p", [2, 3])
def test_cocycles_are_not_coboundaries(p):
    """A bar's cocycle, restricted to the simplices older than its death
    simplex (all of them for an essential class), is not a coboundary there:
    it represents a nonzero class."""
    o = _oracle()
    checked = 0
    for d in _clouds():
        t, res = _with_bars(o, d, 1, p)
        for bar, (idx, cf) in zip(res.bars, res.cocycles):
            if int(bar["dim"]) != 1:
                continue
            edges = _complex(d, 1, t)
            verts = list(_complex(d, 0, t))
            if np.isfinite(bar["death"]):
                ds = int(bar["death_simplex"])
                tris = _complex(d, 2, t)
                tau = next(s for s in tris if _index(s) == ds)
                limit = (tris[tau], ds)
                # edges present when the death simplex enters: no younger than its diameter
                keep = [s for s in edges if edges[s] <= limit[0]]
            else:
                keep = list(edges)
            z = {int(i): int(c) for i, c in zip(idx, cf)}
            restricted = {i: c for i, c in z.items() if any(_index(s) == i for s in keep)}
            assert not _is_coboundary(restricted, verts, keep, p)
            checked += 1
    assert checked > 0


def test_polygon_cocycle_pairs_with_the_polygon():
    """Regular octagon with a threshold between its side and its shorter
    diagonal: the complex is the 8-cycle, H1 has one essential class, and its
    cocycle evaluated on the oriented cycle 0-1-...-7-0 is nonzero."""
    o = _oracle()
    th = np.linspace(0, 2 * np.pi, 8, endpoint=False)
    x = np.stack([np.cos(th), np.sin(th)], 1)
    d = np.sqrt(((x[:, None] - x[None]) ** 2).sum(-1)).astype(np.float32)
    side = float(d[0, 1])
    for p in (2, 3, 5):
        res = o.barcodes(d, 1, side * 1.05, p, cocycles=True)
        h1 = [(b, c) for b, c in zip(res.bars, res.cocycles) if int(b["dim"]) == 1]
        assert len(h1) == 1 and not np.isfinite(h1[0][0]["death"])
        z = {int(i): int(c) for i, c in zip(*h1[0][1])}
        pairing = 0
        for a in range(8):
            b = (a + 1) % 8
            sign = 1 if a < b else -1  # the edge (a, b) is stored oriented from its smaller vertex
            pairing += sign * z.get(_index((a, b)), 0)
        assert pairing % p != 0
