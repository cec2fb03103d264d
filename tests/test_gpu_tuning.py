"""Launch parameters never change a result: the same bars with extreme
settings (every column given to a block at once, or none ever; one block per
SM) as with the defaults, and after the autotuner has installed its choice."""
import math

import numpy as np
import pytest

from paper_1908_02518_gb300 import workloads as W

pytestmark = pytest.mark.gpu

EXTREMES = [
    {"warp_chain_limit": 1, "warp_merge_max": 1},  # every reduced column goes to a block
    {"warp_chain_limit": 1 << 30, "warp_merge_max": 1 << 30},  # warps never give a column up
    {"reduce_blocks_per_sm": 1, "scan_blocks_per_sm": 1},
]


@pytest.fixture(autouse=True)
def _clean_table():
    from paper_1908_02518_gb300 import tuning
    tuning.clear_tuning()
    yield
    tuning.clear_tuning()


def _bars(res):
    b = res.bars
    return sorted(zip(b["cloud"].tolist(), b["dim"].tolist(), b["birth"].tolist(), b["death"].tolist(),
                      b["birth_simplex"].tolist(), b["death_simplex"].tolist()))


CASES = [
    ("torus300", lambda: W.distance_matrix(W.torus_points(300, 21)), 2, 1.2, 2),
    ("s3_48_z3", lambda: W.distance_matrix(W.sphere_points(48, 1005, 4)), 3, math.inf, 3),
]


@pytest.mark.parametrize("name,make,dim_max,t,p", CASES)
@pytest.mark.parametrize("params", EXTREMES)
def test_extreme_settings_give_the_same_bars(name, make, dim_max, t, p, params):
    import torch
    import paper_1908_02518_gb300 as rg
    from paper_1908_02518_gb300 import tuning
    d = torch.from_numpy(make()).cuda()
    want = _bars(rg.barcodes(d, dim_max, t, p))
    n = d.shape[0]
    for dim in range(1, dim_max + 1):
        tuning.set_tuning(dim, 1, 1 << 20, params)
    got = rg.barcodes(d, dim_max, t, p)
    assert _bars(got) == want
    assert got.stats[0][1]["pairs"] >= 0 and n > 0


def test_autotuned_batch_gives_the_same_bars():
    import torch
    import paper_1908_02518_gb300 as rg
    from paper_1908_02518_gb300 import tuning
    clouds = W.batch_clouds(count=16)
    offsets = np.concatenate([[0], np.cumsum([len(c) for c in clouds])]).astype(np.int64)
    pts = torch.from_numpy(np.concatenate(clouds)).cuda()
    want = _bars(rg.barcodes_batched(pts, offsets, 1))
    grid = {"warp_chain_limit": (8, 32), "warp_merge_max": (2048,), "reduce_blocks_per_sm": (0,),
            "scan_blocks_per_sm": (16,)}
    table = tuning.autotune(lambda: rg.barcodes_batched(pts, offsets, 1), max(len(c) for c in clouds), [1],
                            reps=1, grid=grid, budget_s=30)
    assert set(table) == {1}
    assert table[1]["ms"] <= table[1]["default_ms"]
    assert tuning.get_tuning(1, max(len(c) for c in clouds)) == table[1]["params"]
    assert _bars(rg.barcodes_batched(pts, offsets, 1)) == want
