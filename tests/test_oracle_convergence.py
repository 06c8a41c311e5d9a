"""Section 2.3's condition-number argument and Section 2's convergence
statement, measured on the oracle (no GPU).

The paper: the block-Jacobi iteration of Eq. (1) converges at a rate set by
the condition number of H_z^{-1} H, about the square of the horizontal
Courant number nu ~ 10; each coarsening (dx doubled) divides it by 4, so
after three coarsenings it is about nu^2 / 4^3 = 1.56 and four levels
suffice (fixture tests/golden/shallow_multigrid_section_2_3.txt).  Section 2:
a multigrid iteration cuts the residual by about one order of magnitude.

kappa = lambda_max / lambda_min of H_z^{-1} H comes from the oracle's
operator by a Lanczos solve (oracle.hz_spectrum), on bands of rows with
zero-flux edges so that the equator and the pole rows are seen apart; nu^2
is read off lambda_min (oracle.courant_squared: (1/lambda_min - 1) / 4 on
square cells).  The grid is 2:1 (square cells at the equator), two layers
(H_z^{-1} removes the vertical: the values do not change with nz).
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import tpmg as O
from synthetic import make_problem
from test_golden_paper import read_fixture


def _band_rows(lev, which):
    deg = np.degrees(lev.centres)
    if which == "equator":
        rows = np.where(np.abs(deg) < 12.0)[0]
        return rows[0], rows[-1] + 1
    return lev.nlat - 6, lev.nlat            # the six rows next to the north pole


@pytest.fixture(scope="module")
def spectra():
    """(lambda_min, lambda_max) per level for both bands of a 512 x 256 x 2
    grid on the four levels of Section 2.3's shallow hierarchy."""
    P = make_problem(512, 256, 2, 0.1, 1000)
    lev = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], O.MGParams(levels=4))
    out = {"equator": [], "pole": []}
    for L in lev:
        for which in out:
            j0, j1 = _band_rows(L, which)
            out[which].append(O.hz_spectrum(O.row_band(L, j0, j1), tol=1e-6))
    return out


def test_spectrum_matches_dense_generalised_eigenproblem():
    """The Lanczos routine and the probed sparse operator against the dense
    operator (built column by column from unit vectors) and LAPACK's
    generalised symmetric eigensolver, on 8 x 4 x 4."""
    P = make_problem(8, 4, 4, 0.2, 3)
    lev = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], O.MGParams(levels=1))[0]
    A = O.dense_operator(lev)
    assert np.array_equal(O.sparse_operator(lev).toarray(), A)
    ncol = lev.nlat * lev.nlon
    idx = np.arange(lev.size)
    same_column = (idx[:, None] % ncol) == (idx[None, :] % ncol)
    ev = scipy.linalg.eigh(A, np.where(same_column, A, 0.0), eigvals_only=True)
    lmin, lmax = O.hz_spectrum(lev)
    assert lmin == pytest.approx(ev[0], rel=1e-8)
    assert lmax == pytest.approx(ev[-1], rel=1e-8)


def test_spectrum_bounds(spectra):
    """Bounds that hold for any such operator: 2 H_z - H = H_z - dH is
    positive definite (diagonal dominance with h > 0), so lambda_max < 2;
    lambda_min is at most the Rayleigh quotient of the constant vector,
    sum h / sum (h + horizontal couplings) on a band with zero-flux edges."""
    P = make_problem(64, 32, 4, 0.2, 5)
    lev = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], O.MGParams(levels=1))[0]
    band = O.row_band(lev, 10, 22)
    lmin, lmax = O.hz_spectrum(band)
    one = np.ones(band.shape)
    # 1' H 1 = sum h (H 1 = h); 1' H_z 1 = sum (h + horizontal couplings)
    rq = O.dot(one, O.apply(band, one)) / float(np.sum(band.h + _horizontal(band)))
    assert 0 < lmin <= rq and lmax < 2.0
    for which in spectra:
        assert all(0 < a < b < 2.0 for a, b in spectra[which])


def _horizontal(lev):
    """Sum of the four horizontal couplings of every cell."""
    tx, ty = lev.tx, lev.ty
    s = tx + np.roll(tx, 1, axis=2) + ty
    s[:, 1:, :] += ty[:, :-1, :]
    return s


def test_section_2_3_law_at_the_equator(spectra):
    """Where the paper's premise holds (cells of aspect ~1, nu ~ 10): nu^2
    read off the spectrum is ~100 on the finest level, each coarsening
    divides kappa by ~4, and after three coarsenings nu^2 is ~1.56 (the
    printed figure).  Measured: nu^2 98.1, 24.2, 5.84, 1.37; kappa 785, 195,
    47.7, 11.9."""
    g = read_fixture("shallow_multigrid_section_2_3.txt")
    nu2 = g["courant_number"] ** 2
    lam = spectra["equator"]
    kappa = [b / a for a, b in lam]
    c2 = [O.courant_squared(a) for a, _ in lam]
    print("equator: kappa", ["%.4g" % k for k in kappa], "nu^2", ["%.4g" % c for c in c2])
    assert len(lam) == int(g["levels"])
    for l, c in enumerate(c2):
        assert c == pytest.approx(nu2 / g["reduction_per_coarsening"] ** l, rel=0.2)
    for a, b in zip(kappa, kappa[1:]):
        assert 3.0 <= a / b <= 5.0
    assert c2[int(g["coarsenings"])] == pytest.approx(g["condition_number_after"], rel=0.2)


def test_section_2_3_law_breaks_at_the_pole_rows(spectra):
    """On the lat-lon grid the longitude couplings grow as 1/cos^2(theta)
    towards the poles.  Conditional semi-coarsening keeps dividing kappa by
    ~4 there (longitude is halved on every level), but from a start ~1/cos^2
    of the first row (~2.7e4 at 256 rows) above nu^2: after three
    coarsenings nu^2 is still ~1.2e3, hundreds of times the 1.56 that makes
    four levels enough.  Measured: nu^2 7.7e4, 1.9e4, 4.8e3, 1.2e3."""
    g = read_fixture("shallow_multigrid_section_2_3.txt")
    lam = spectra["pole"]
    kappa = [b / a for a, b in lam]
    c2 = [O.courant_squared(a) for a, _ in lam]
    print("pole rows: kappa", ["%.4g" % k for k in kappa], "nu^2", ["%.4g" % c for c in c2])
    for a, b in zip(kappa, kappa[1:]):
        assert 3.0 <= a / b <= 5.0
    assert c2[int(g["coarsenings"])] >= 100 * g["condition_number_after"]
    assert c2[0] >= 100 * g["courant_number"] ** 2


def _mean_reduction(hist):
    return (hist[-1] / hist[0]) ** (1.0 / (len(hist) - 1))


def test_one_order_of_magnitude_per_iteration():
    """Section 2: each multigrid iteration reduces the residual norm by about
    one order of magnitude.  Reached by the V(2,2)-cycle as the
    preconditioner of conjugate gradients on the default hierarchy (measured
    0.109 per iteration on 64 x 32 x 16); V(3,3) goes further."""
    P = make_problem(64, 32, 16, 0.1, 1000)
    for nu, lo, hi in ((2, 0.05, 0.15), (3, 0.03, 0.1)):
        p = O.MGParams(nu1=nu, nu2=nu)
        lev = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], p)
        _, hist, st = O.solve(lev, P["b"], 1e-10, params=p)
        assert st == O.OK
        assert lo <= _mean_reduction(hist) <= hi, (nu, _mean_reduction(hist))


def test_vcycle_1_1_rate_is_set_by_the_smoother():
    """Why V(1,1) does not reach 0.1 on its own: with the coarse problem
    solved exactly (two levels, the coarse level by 150 PCG iterations) the
    stationary V(1,1) still contracts the error by only ~0.46 per cycle (V(2,2)
    ~0.24), so
    neither the depth of the hierarchy nor the coarse solve sets the rate.
    Damped Jacobi on the horizontal couplings reduces the highest
    frequencies by |1 - 2 omega| (0.6 at the best omega = 0.8 on square
    cells) per sweep, ~0.36 for two sweeps; V(2,2) roughly squares the
    V(1,1) factor."""
    P = make_problem(64, 32, 16, 0.1, 1000)
    rates = []
    for nu in (1, 2):
        p = O.MGParams(nu1=nu, nu2=nu, omega=0.8, levels=2, coarse_method="pcg",
                       coarse_iters=150, method="stationary")
        lev = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], p)
        x = np.random.default_rng(0).standard_normal(lev[0].shape)
        zero = np.zeros_like(x)
        hist = []
        for _ in range(30):  # past the fast start: the asymptotic rate
            r = O.residual(lev[0], zero, x)
            hist.append(O.norm2(r))
            x += O.vcycle(lev, r, p)
        rates.append((hist[-1] / hist[-11]) ** 0.1)
    print("two-grid stationary rates V(1,1), V(2,2):", rates)
    assert 0.35 <= rates[0] <= 0.6
    assert rates[1] <= 1.2 * rates[0] ** 2


def test_isotropy_stopping_rule():
    """levels = -1 stops at the first level whose largest (sum of horizontal
    couplings) / h is within iso_ratio (Section 2.3's premise for stopping:
    the coarse problem is well conditioned).  On the lat-lon sphere the pole
    rows never get there before the depth limit (their ratio falls 4x per
    level from ~850: 849, 213, 56, 15, 0.65 even with a Helmholtz term 100
    times larger); with one 10^4 times larger it stops after one
    coarsening."""
    P = make_problem(64, 32, 16, 0.1, 1000)
    deep = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], O.MGParams())
    iso = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], O.MGParams(levels=-1))
    assert len(iso) == len(deep)
    assert all(O.horizontal_ratio(L) > 6.25 for L in iso)
    h = P["h"] * 1e4
    p = O.MGParams(levels=-1)
    lev = O.build_hierarchy(P["tx"], P["ty"], P["tz"], h, p)
    ratios = [O.horizontal_ratio(L) for L in lev]
    print("ratios per level with h x 1e4:", ratios)
    assert 1 < len(lev) < len(deep)
    assert ratios[-1] <= p.iso_ratio and all(r > p.iso_ratio for r in ratios[:-1])
    x, hist, st = O.solve(lev, P["b"], 1e-10, params=p)
    assert st == O.OK
