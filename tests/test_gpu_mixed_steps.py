"""Error of the mixed-precision solve against the oracle's FP64 solution
after each refinement step (the precision form's report), on a 512 x 384 x 70
grid with the workload generator (sigma 0.1).  The 1024 x 768 x 70 grid the
report is named for takes the CPU oracle about a minute per solve on the GPU
host; this grid keeps the same level structure (8 levels, 70 layers) at a
quarter of the cost.

Bounds from the oracle's own mixed solve of this system (its per-step errors
1.4e-4, 4.5e-8, 9.8e-12): each FP32 inner solve gains at most about four
orders (its attainable accuracy), so one, two and three steps must be within
1e-3, 1e-6 and 1e-10, each at least 100 times better than the one before.
"""
import numpy as np
import pytest

from gpu_common import dev, handle_for, host, oracle_levels, problem, rel_2
from oracle import tpmg as O

pytestmark = pytest.mark.gpu


def test_mixed_error_after_each_refinement_step():
    P = problem(512, 384, 70, sigma=0.1, seed=2000)
    lev, p = oracle_levels(P)
    xs, _, st = O.solve(lev, P["b"], 1e-12, params=p)
    assert st == O.OK
    errs = []
    for steps in (1, 2, 3):
        H = handle_for(P, maxit=steps)
        x, info = H.solve_mixed(dev(P["b"]), tol=1e-10, raise_on_error=False)
        assert info["iterations"] == steps
        errs.append(rel_2(host(x), xs))
        del H
    print("mixed-precision error after 1, 2, 3 refinement steps:",
          ", ".join("%.2e" % e for e in errs))
    assert errs[0] <= 1e-3 and errs[1] <= 1e-6 and errs[2] <= 1e-10
    assert errs[1] <= 1e-2 * errs[0] and errs[2] <= 1e-2 * errs[1]
