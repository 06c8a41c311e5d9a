"""Error of the mixed-precision solve against the oracle's FP64 solution
after each refinement step (the precision form's report), on the
1024 x 768 x 70 workload itself (seed 2000, sigma 0.1).

The GPU's errors are printed beside the oracle's own mixed solve of the same
system (the oracle's float V-cycle inside its FP64 refinement); measured:
GPU 2.0e-3, 7.1e-8, 6.8e-11 and oracle 2.0e-3, 2.5e-8, 5.9e-12.  The first
FP32 inner solve stops at its relative residual tolerance of 5e-4, and the
error of the iterate is a few times its residual on this operator (~4 here),
so one step must be within 5e-3; each further step gains at least two and at
most about four orders of magnitude (the attainable accuracy of a
single-precision solve), so two and three steps must be within 1e-6 and
1e-10, each at least 100 times better than the one before.  The GPU and
oracle trajectories differ only by FP32 rounding order, so the GPU's first
two errors stay within a factor 30 of the oracle's.
"""
import numpy as np
import pytest

from gpu_common import dev, handle_for, host, oracle_levels, rel_2
from oracle import tpmg as O
from synthetic import WORKLOADS, make_problem, workload_seed

pytestmark = pytest.mark.gpu

WORKLOAD = "latlon_1024x768x70"


def test_mixed_error_after_each_refinement_step():
    w = WORKLOADS[WORKLOAD]
    P = make_problem(w["nlon"], w["nlat"], w["nz"], w["sigma"], workload_seed(WORKLOAD))
    lev, p = oracle_levels(P)
    xs, _, st = O.solve(lev, P["b"], 1e-12, params=p)
    assert st == O.OK
    orc = []
    O.solve_mixed(lev, P["b"], 1e-10, params=p, maxit=3,
                  track=lambda x: orc.append(rel_2(x, xs)))
    errs = []
    for steps in (1, 2, 3):
        H = handle_for(P, maxit=steps)
        x, info = H.solve_mixed(dev(P["b"]), tol=1e-10, raise_on_error=False)
        assert info["iterations"] == steps
        errs.append(rel_2(host(x), xs))
        del H
    print(f"{WORKLOAD}: mixed-precision error after 1, 2, 3 refinement steps: GPU",
          ", ".join("%.2e" % e for e in errs), "| oracle", ", ".join("%.2e" % e for e in orc))
    assert errs[0] <= 5e-3 and errs[1] <= 1e-6 and errs[2] <= 1e-10
    assert errs[1] <= 1e-2 * errs[0] and errs[2] <= 1e-2 * errs[1]
    for g, o in zip(errs[:2], orc[:2]):
        assert g <= 30 * o and o <= 30 * g
