"""BiCGStab of the oracle (Section 1: the ENDGame solver the multigrid
replaced, BiCGStab preconditioned by the vertical line relaxation of
Eq. (1); and its V-cycle-preconditioned variant), pinned without the GPU.

* converged solutions against the dense row-sum LU solve;
* the first iteration against the same step assembled by hand from dense
  matrices (H column by column from unit vectors; the preconditioner of one
  sweep from zero is omega H_z^{-1}, H_z the same-column part of H);
* Section 1's single-precision remark: in FP32 the line-relaxed BiCGStab
  loses its convergence (its residual ends above where it started), while
  the multigrid iteration settles at the FP32 floor of the operator and
  stays there.
"""
import numpy as np
import pytest

from oracle import tpmg as O
from synthetic import make_problem
from test_oracle_pins import _dense_solve, levels_of


@pytest.mark.parametrize("method", ["bicgstab_line", "bicgstab"])
@pytest.mark.parametrize("shape", [(8, 4, 4), (16, 8, 6)])
def test_bicgstab_matches_dense_lu(shape, method):
    P = make_problem(*shape, 0.1, 11)
    lev, p = levels_of(P, method=method, maxit=2000)
    x, hist, st = O.solve(lev, P["b"], 1e-13, params=p)
    xd, _ = _dense_solve(P, P["b"])
    # the residual floor of these tiny grids is ~1e-11: compare solutions
    assert st in (O.OK, O.NOT_CONVERGED)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def test_first_iteration_assembled_by_hand():
    """One BiCGStab iteration from x = 0 with M = omega H_z^{-1}."""
    P = make_problem(8, 4, 4, 0.2, 12)
    lev, p = levels_of(P, method="bicgstab_line", line_sweeps=1)
    A = O.dense_operator(lev[0])
    n = A.shape[0]
    idx = np.arange(n)
    ncol = lev[0].nlat * lev[0].nlon
    Z = np.where((idx[:, None] % ncol) == (idx[None, :] % ncol), A, 0.0)
    M = p.omega * np.linalg.inv(Z)
    b = P["b"].ravel()
    r = b.copy()
    rh = b.copy()
    rho = rh @ r
    pv = r
    ph = M @ pv
    v = A @ ph
    alpha = rho / (rh @ v)
    s = r - alpha * v
    sh = M @ s
    t = A @ sh
    w = (t @ s) / (t @ t)
    x1 = alpha * ph + w * sh
    x, hist, st = O.solve_bicgstab(lev, P["b"], 1e-30, p, maxit=1, precond="line")
    # history: the start, the recursive residual after the iteration, and
    # the true residual of x1 that the stop confirms
    assert st == O.NOT_CONVERGED and len(hist) == 3
    assert np.linalg.norm(x.ravel() - x1) <= 1e-12 * np.linalg.norm(x1)
    r1 = s - w * t
    rel1 = np.linalg.norm(r1) / np.linalg.norm(b)
    assert hist[1] == pytest.approx(rel1, rel=1e-10)
    assert hist[2] == pytest.approx(np.linalg.norm(b - A @ x1) / np.linalg.norm(b), rel=1e-8)


def test_line_relaxation_is_omega_hz_inverse_for_one_sweep():
    P = make_problem(16, 8, 5, 0.2, 13)
    lev, p = levels_of(P)
    r = np.random.default_rng(0).standard_normal(lev[0].shape)
    got = O.line_relaxation(lev[0], r, 1, p.omega)
    assert np.allclose(got, p.omega * O.column_solve(lev[0], r), rtol=1e-14, atol=0)


def test_bicgstab_iterations_grow_with_resolution_multigrid_does_not():
    """Line-relaxed BiCGStab needs more iterations as the grid is refined
    (the pole rows' condition number grows as 1/cos^2 of the first row,
    ~nlat^2), the V-cycle-preconditioned solvers stay flat."""
    its = {}
    for shape in ((64, 32, 8), (128, 64, 8)):
        P = make_problem(*shape, 0.1, 1000)
        for m in ("bicgstab_line", "bicgstab", "cg"):
            lev, p = levels_of(P, method=m, maxit=3000)
            _, hist, st = O.solve(lev, P["b"], 1e-8, params=p)
            assert st == O.OK
            its[(shape, m)] = len(hist) - 1
    print(its)
    assert its[((128, 64, 8), "bicgstab_line")] >= 1.6 * its[((64, 32, 8), "bicgstab_line")]
    for m in ("bicgstab", "cg"):
        assert abs(its[((128, 64, 8), m)] - its[((64, 32, 8), m)]) <= 2
        assert its[((128, 64, 8), m)] * 10 < its[((128, 64, 8), "bicgstab_line")]


def test_single_precision_bicgstab_loses_convergence_multigrid_does_not():
    """Section 1: run in single precision, the Krylov solver struggles at
    tight tolerances.  On the FP32 hierarchy (FP32 storage and arithmetic,
    FP64 inner products) with a tolerance below the FP32 floor, 300
    iterations: the line-relaxed BiCGStab's residual ends above its start;
    the V-cycle-preconditioned CG's true residual sits at the FP32 floor
    (~2.5e-3 here, the rounding of x times couplings ~1e6 h) and its last
    restart is no worse than its best."""
    P = make_problem(64, 32, 16, 0.1, 2000)
    b = P["b"]
    out = {}
    for m in ("bicgstab_line", "cg"):
        lev, p = levels_of(P, method=m, maxit=300)
        l32 = O.float_levels(lev)
        s = float(np.ldexp(1.0, int(np.frexp(np.max(np.abs(b)))[1])))
        x32, hist, st = O.solve(l32, (b / s).astype(np.float32), 1e-10, params=p)
        x = (l32[0].scale * s) * x32.astype(np.float64)
        true = O.norm2(O.residual(lev[0], b, x)) / O.norm2(b)
        out[m] = (st, np.array(hist), true)
    st, h, true = out["bicgstab_line"]
    assert st == O.NOT_CONVERGED and h[-1] > 1.0 and true > 1.0
    st, h, true = out["cg"]
    assert st == O.NOT_CONVERGED and true <= 1e-2
    assert true <= 2 * out["bicgstab_line"][1].min()
