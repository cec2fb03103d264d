"""Backward pass: gradients of loss = sum over H1 bars of (death - birth)^2 with
respect to the point coordinates, against (a) the float64 reference gradient
from the oracle's pairs and (b) float64 central finite differences with step
1e-4 (coordinates whose pairing changes within +-h are skipped and counted).
Tolerance: ||g - g_ref||_inf <= 1e-4 * max(||g_ref||_inf, 1e-6)."""
import numpy as np
import pytest

from paper_1908_02518_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-4
STEP = 1e-4


def _gpu_grad(clouds, dim_max=1):
    import torch
    import paper_1908_02518_gb300 as rg
    off = np.concatenate([[0], np.cumsum([c.shape[0] for c in clouds])]).astype(np.int64)
    x = torch.from_numpy(np.concatenate(clouds)).cuda().requires_grad_(True)
    birth, death, dim, cloud = rg.RipsBarcodes.apply(x, off.tolist(), dim_max)
    fin = torch.isfinite(death) & (dim == 1)
    loss = ((death - birth)[fin] ** 2).sum()
    loss.backward()
    return x.grad.double().cpu().numpy(), float(loss), off


def _ref_grad(pts, oracle_mod):
    from oracle import gradients as G
    d32 = G.distances32(pts)
    r = oracle_mod.barcodes(d32, 1)
    bars = r.dim(1)
    bars = bars[np.isfinite(bars["death"])]
    diff = (bars["death"].astype(np.float64) - bars["birth"].astype(np.float64))
    return G.bar_gradient(pts, bars, -2 * diff, 2 * diff)


def _pairs(pts64, oracle_mod):
    from oracle import gradients as G
    d32 = G.distances32(pts64)
    r = oracle_mod.barcodes(d32, 1)
    bars = r.dim(1)
    bars = bars[np.isfinite(bars["death"])]
    key = tuple(sorted((int(b["birth_simplex"]), int(b["death_simplex"])) for b in bars))
    return key, G.endpoint_edges(d32, bars)


def _fd_grad(pts, oracle_mod, coords=None):
    from oracle import gradients as G
    x0 = np.asarray(pts, dtype=np.float32).astype(np.float64)
    base, _ = _pairs(x0, oracle_mod)
    g = np.full(x0.shape, np.nan)
    skipped = 0
    idx = coords if coords is not None else [(i, c) for i in range(x0.shape[0]) for c in range(x0.shape[1])]
    for i, c in idx:
        vals = []
        ok = True
        for s in (+1, -1):
            x = x0.copy()
            x[i, c] += s * STEP
            key, edges = _pairs(x, oracle_mod)
            if key != base:
                ok = False
                break
            vals.append(G.h1_loss(x, edges))
        if not ok:
            skipped += 1
            continue
        g[i, c] = (vals[0] - vals[1]) / (2 * STEP)
    return g, skipped


def _close(g, ref):
    m = ~np.isnan(ref)
    err = np.abs(g[m] - ref[m]).max() if m.any() else 0.0
    scale = max(np.abs(ref[m]).max() if m.any() else 0.0, 1e-6)
    return err <= TOL * scale, err, scale


@pytest.mark.parametrize("kind", ["circle", "torus", "cube"])
def test_gradient_matches_reference_and_fd(oracle_mod, kind):
    rng = np.random.Generator(np.random.PCG64(700 + len(kind)))
    n = 40
    if kind == "circle":
        pts = W.circle_points(rng, n, 0.05).astype(np.float32)
    elif kind == "torus":
        pts = W._torus(rng, n, 2.0, 1.0, 0.02).astype(np.float32)
    else:
        pts = rng.random((n, 3)).astype(np.float32)
    g, loss, _ = _gpu_grad([pts])
    ref = _ref_grad(pts, oracle_mod)
    ok, err, scale = _close(g, ref)
    assert ok, (err, scale)
    fd, skipped = _fd_grad(pts, oracle_mod)
    assert skipped <= pts.size // 10
    ok, err, scale = _close(g, fd)
    assert ok, (err, scale, skipped)


def test_batched_gradient_matches_reference(oracle_mod):
    clouds = W.batch_clouds(count=12, lo=64, hi=160, meta_seed=4100, cloud_seed=41000)
    g, _, off = _gpu_grad(clouds)
    for c, pts in enumerate(clouds):
        ref = _ref_grad(pts, oracle_mod)
        ok, err, scale = _close(g[off[c]:off[c + 1]], ref)
        assert ok, (c, err, scale)


def test_grad_dist_scatter(oracle_mod):
    """dL/dD through the C ABI equals the per-bar sum on the critical edges."""
    import torch
    import paper_1908_02518_gb300 as rg
    from oracle import gradients as G
    pts = W.cube_points(30, 77)
    x = torch.from_numpy(pts).cuda()
    res = rg.barcodes_batched(x, [0, 30], 1, keep_handle=True)
    nb = len(res.bars)
    gb = torch.arange(nb, dtype=torch.float32, device="cuda") * 0.01
    gd = torch.ones(nb, dtype=torch.float32, device="cuda")
    gD = torch.zeros(30 * 30, dtype=torch.float32, device="cuda")
    rg.backward(res, x, gb, gd, grad_dist=gD)
    want = np.zeros((30, 30))
    d32 = G.distances32(pts)
    for q, (be, de) in enumerate(G.endpoint_edges(d32, res.bars.astype(
            [("dim", "i4"), ("birth", "f4"), ("death", "f4"), ("cloud", "i4"), ("birth_simplex", "i8"),
             ("death_simplex", "i8")]))):
        if be is not None:
            want[be] += 0.01 * q
        if de is not None:
            want[de] += 1.0
    np.testing.assert_allclose(gD.view(30, 30).cpu().numpy(), want, rtol=1e-6, atol=1e-6)
