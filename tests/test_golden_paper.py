"""The oracle against numbers the paper prints (fixtures in tests/golden/,
each citing its passage)."""
import os

import numpy as np
import pytest

from oracle import tpmg as O
from synthetic import make_problem

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def read_fixture(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                key, val = line.split()
                vals[key] = float(val)
    return vals


@pytest.mark.parametrize("shape", [(256, 128, 8), (1536, 1152, 4)])
def test_shallow_multigrid_condition_number(shape):
    """Section 2.3: with nu ~ 10 on the finest grid, each coarsening divides
    the horizontal-to-Helmholtz coupling ratio (the condition number of the
    column iteration, ~ nu^2) by 4, reaching ~1.56 after three coarsenings,
    on the fourth and last level of the shallow hierarchy.  Measured at the
    equatorial row of the lowest layer (radius within 0.3 % of the planet's)
    as (t_x / h) cos^2(theta), which removes the sphere's 1/cos^2 longitude
    metric; this exercises the synthetic coefficients
    (K = (nu R dlambda)^2), the coarse Helmholtz sums and the rescaling of
    the coarse longitude couplings by the fine/coarse centre distances."""
    g = read_fixture("shallow_multigrid_section_2_3.txt")
    P = make_problem(*shape, 0.0, 0)
    lev = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"],
                            O.MGParams(levels=int(g["levels"])))
    assert len(lev) == int(g["levels"]) == int(g["coarsenings"]) + 1
    nu2 = g["courant_number"] ** 2
    for l, f in enumerate(lev):
        j = f.nlat // 2
        k = 0
        ratio = f.tx[k, j, 0] / f.h[k, j, 0] * np.cos(f.centres[j]) ** 2
        want = nu2 / g["reduction_per_coarsening"] ** l
        assert ratio == pytest.approx(want, rel=0.02)
    assert abs(ratio - g["condition_number_after"]) <= 0.01  # printed to two decimals
