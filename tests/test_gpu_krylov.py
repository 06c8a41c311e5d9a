"""BiCGStab on the GPU (the solver of Section 1 that the multigrid replaced:
BiCGStab preconditioned by the vertical line relaxation of Eq. (1); and its
V-cycle-preconditioned form) against the oracle, and the whole solve in
single precision (Section 1's single-precision remark).

FP64 solutions solved to 5e-12 on both sides agree to 1e-10 relative;
iteration counts agree within rounding (10 %, at least 3).  In single
precision the multigrid solution is accurate to FP32 rounding (the oracle's
FP32 solve gives 4.6e-8 relative error on 64 x 32 x 16, although its FP64
residual stalls near 1.4e-3: the rounding of x times the vertical couplings),
while the line-relaxed BiCGStab loses its convergence.
"""
import numpy as np
import pytest
import torch

from gpu_common import dev, handle_for, host, oracle_levels, problem, rel_2
from oracle import tpmg as O

pytestmark = pytest.mark.gpu

METHOD = {"bicgstab_line": 3, "bicgstab": 2, "cg": 0}


@pytest.mark.parametrize("method", ["bicgstab_line", "bicgstab"])
@pytest.mark.parametrize("shape", [(64, 32, 16), (96, 46, 9)])
def test_bicgstab_fp64_matches_oracle(shape, method):
    P = problem(*shape, sigma=0.2, seed=sum(shape))
    lev, p = oracle_levels(P, method=method, maxit=4000)
    xr, hr, st = O.solve(lev, P["b"], 5e-12, params=p)
    assert st == O.OK
    H = handle_for(P, method=METHOD[method], maxit=4000, mixed=0)
    x, info = H.solve(dev(P["b"]), tol=5e-12)
    assert info["status"] == 0 and info["rel_res"] <= 5e-12
    assert rel_2(host(x), xr) <= 1e-10
    its_o = len(hr) - 1
    assert abs(info["iterations"] - its_o) <= max(3, 0.1 * its_o), (info["iterations"], its_o)


def test_bicgstab_inside_mixed_refinement():
    """The V-cycle-preconditioned BiCGStab as the FP32 inner solver of the
    mixed-precision refinement reaches the FP64 solution."""
    P = problem(96, 46, 12, sigma=0.2, seed=77)
    lev, p = oracle_levels(P)
    xr, _, _ = O.solve(lev, P["b"], 1e-12, params=p)
    H = handle_for(P, method=METHOD["bicgstab"])
    x, info = H.solve_mixed(dev(P["b"]), tol=1e-10)
    assert info["status"] == 0 and info["rel_res"] <= 1e-10
    assert rel_2(host(x), xr) <= 1e-9


def test_single_precision_multigrid_solve():
    """mg_solve_single with the default method: its FP32 residual history
    agrees with the oracle's FP32 solve over the first iterations, and the
    solution reaches FP32 accuracy (a tolerance below the FP32 floor ends
    NOT_CONVERGED)."""
    P = problem(64, 32, 16, sigma=0.2, seed=112)
    lev, p = oracle_levels(P, maxit=60)
    xr, _, _ = O.solve(lev, P["b"], 1e-12)
    l32 = O.float_levels(lev)
    b = P["b"]
    b32 = b.astype(np.float32)
    _, ho, _ = O.solve(l32, b32, 1e-10, params=p)
    H = handle_for(P, maxit=60)
    x32, info = H.solve_single(dev(b32, torch.float32), tol=1e-10, raise_on_error=False)
    assert info["status"] == 4  # MG_ERR_NOT_CONVERGED: below the FP32 floor
    x = host(x32).astype(np.float64)
    assert rel_2(x, xr) <= 1e-6
    true = O.norm2(O.residual(lev[0], b, x)) / O.norm2(b)
    assert true <= 5e-3
    # the residuals carry FP32 rounding of ~1e-3 of ||b|| (the floor above):
    # the first steps agree to that
    assert len(info["history"]) >= 3
    for g, o in zip(info["history"][:3], ho[:3]):
        assert abs(g - o) <= 3e-3


def test_single_precision_line_bicgstab_loses_convergence():
    """Section 1: in single precision the line-relaxed BiCGStab does not
    converge (its residual ends far above its best and its solution is
    worse than the FP32 multigrid's by orders of magnitude)."""
    P = problem(64, 32, 16, sigma=0.1, seed=2000)
    lev, _ = oracle_levels(P)
    xr, _, _ = O.solve(lev, P["b"], 1e-12)
    b32 = dev(P["b"].astype(np.float32), torch.float32)
    out = {}
    for m in ("bicgstab_line", "cg"):
        H = handle_for(P, method=METHOD[m], maxit=300)
        x32, info = H.solve_single(b32, tol=1e-10, raise_on_error=False)
        out[m] = (info, rel_2(host(x32).astype(np.float64), xr))
    info, err = out["bicgstab_line"]
    assert info["status"] in (4, 5)  # not converged or diverged
    assert err >= 1e3 * out["cg"][1]
    assert out["cg"][1] <= 1e-6


def test_batch_rejects_bicgstab():
    from paper_2307_04528_gb300 import _lib as L
    from paper_2307_04528_gb300.solver import MGBatch
    P = problem(32, 16, 4, sigma=0.1, seed=5)
    systems = [tuple(dev(P[k]) for k in ("tx", "ty", "tz", "h"))]
    with pytest.raises(L.MGError) as e:
        MGBatch(systems, method=METHOD["bicgstab"])
    assert e.value.status == L.MG_ERR_ARG
