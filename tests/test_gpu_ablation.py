"""The ablation switches of Table 3: the apparent-pair skip and the emergent
first-pivot shortcut turned off, alone and together.  The barcode must not
change (bar by bar against the oracle), and the Table-2 counters must show
what each shortcut did: no apparent pairs without the apparent skip, every
column that is not cleared reduced, the same pairs and essential classes."""
import math

import numpy as np
import pytest

from paper_1908_02518_gb300 import workloads as W

pytestmark = pytest.mark.gpu

U64MAX = int(np.iinfo(np.uint64).max)


def _key(bars):
    return sorted((int(b["dim"]), float(b["birth"]), float(b["death"]), int(b["birth_simplex"]),
                   U64MAX if int(b["death_simplex"]) < 0 else int(b["death_simplex"])) for b in bars)


CASES = [("cube", lambda: W.distance_matrix(W.cube_points(60, 71)), 2, math.inf, 2),
         ("torus", lambda: W.distance_matrix(W.torus_points(150, 72)), 2, 1.2, 2),
         ("ties", lambda: W.random_integer_matrix(18, 73, levels=3), 3, math.inf, 3),
         ("sphere", lambda: W.distance_matrix(W.sphere_points(36, 74)), 3, math.inf, 3)]


@pytest.mark.parametrize("name,make,dim_max,t,p", CASES, ids=[c[0] for c in CASES])
def test_switches_keep_the_barcode(oracle_mod, name, make, dim_max, t, p):
    import torch
    import paper_1908_02518_gb300 as rg
    d = make()
    want = _key(oracle_mod.barcodes(d, dim_max, t, p).bars)
    dev = torch.from_numpy(d).cuda()
    base = rg.barcodes(dev, dim_max, t, p)
    assert _key(base.bars) == want
    try:
        for apparent, emergent in [(False, True), (True, False), (False, False)]:
            rg.set_options(apparent=apparent, emergent=emergent)
            assert rg.get_options() == {"apparent": apparent, "emergent": emergent}
            got = rg.barcodes(dev, dim_max, t, p)
            assert _key(got.bars) == want, (apparent, emergent)
            for k in range(1, dim_max + 1):
                s, b = got.stats[0][k], base.stats[0][k]
                assert s["simplices"] == b["simplices"]
                assert s["essential"] == b["essential"]
                assert s["pairs"] + s["apparent_cofacet"] == b["pairs"] + b["apparent_cofacet"]
                if not apparent:
                    assert s["apparent_cofacet"] == 0 and s["apparent_facet"] == 0
                    assert s["columns"] == s["simplices"] - s["cleared"]
    finally:
        rg.set_options()
