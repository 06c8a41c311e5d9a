"""The Chebyshev coarsest-level solve of the oracle (Section 2.3's simple
coarsest-grid iteration, polynomially accelerated), pinned without the GPU:

* its error after m steps is the Chebyshev polynomial
  T_m((theta - lambda) / delta) / T_m(sigma) of H_z^{-1} H applied to the
  initial error (the closed form of the iteration), evaluated through a
  dense generalised eigendecomposition (LAPACK), on 8 x 4 x 4;
* the interval [mu, 2] it is built on holds the spectrum of H_z^{-1} H
  (dense eigenvalues);
* a V-cycle with it stays a fixed symmetric positive linear operator.
"""
import numpy as np
import pytest
import scipy.linalg

from oracle import tpmg as O
from synthetic import make_problem
from test_oracle_pins import levels_of


def _level(seed, shape=(8, 4, 4)):
    P = make_problem(*shape, 0.2, seed)
    return O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], O.MGParams(levels=1))[0]


def _dense_pair(lev):
    A = O.dense_operator(lev)
    idx = np.arange(A.shape[0])
    ncol = lev.nlat * lev.nlon
    Z = np.where((idx[:, None] % ncol) == (idx[None, :] % ncol), A, 0.0)
    return A, Z


@pytest.mark.parametrize("seed", [3, 4])
def test_interval_holds_the_spectrum(seed):
    lev = _level(seed)
    A, Z = _dense_pair(lev)
    ev = scipy.linalg.eigh(A, Z, eigvals_only=True)
    mu, lam = O.hz_interval(lev)
    assert mu <= ev[0] and ev[-1] < lam
    # the bound is the smallest per-cell ratio: attained only by a constant
    # mode on a uniform level, so it lies below the true minimum here
    assert mu >= 0.05 * ev[0]


@pytest.mark.parametrize("m", [1, 2, 3, 6])
def test_error_is_the_chebyshev_polynomial(m):
    lev = _level(7)
    A, Z = _dense_pair(lev)
    b = np.random.default_rng(m).standard_normal(lev.shape)
    xs = np.linalg.solve(A, b.ravel())
    x = O.coarse_chebyshev(lev, b, m).ravel()
    mu, lam = O.hz_interval(lev)
    theta, delta = 0.5 * (lam + mu), 0.5 * (lam - mu)
    ev, V = scipy.linalg.eigh(A, Z)          # V' Z V = I, (Z^{-1} A) V = V diag(ev)
    T = lambda t: np.polynomial.chebyshev.chebval(t, [0] * m + [1])
    p = T((theta - ev) / delta) / T(theta / delta)
    e_model = V @ (p * (V.T @ (Z @ xs)))     # p(Z^{-1} A) applied to e_0 = x*
    e = xs - x
    assert np.linalg.norm(e - e_model) <= 1e-10 * np.linalg.norm(xs)
    # and it is a contraction: |p| <= 1 / T_m(sigma) on the interval
    assert np.max(np.abs(p)) <= 1.0 / T(theta / delta) * (1 + 1e-12)


def test_vcycle_with_chebyshev_coarse_solve_is_symmetric_linear():
    P = make_problem(32, 16, 8, 0.1, 5)
    lev, p = levels_of(P, levels=3, coarse_method="chebyshev", coarse_iters=8)
    rng = np.random.default_rng(5)
    r1, r2 = rng.standard_normal((2,) + lev[0].shape)
    v1, v2 = O.vcycle(lev, r1, p), O.vcycle(lev, r2, p)
    a, b = O.dot(v1, r2), O.dot(r1, v2)
    assert abs(a - b) <= 1e-12 * abs(a)
    assert O.dot(v1, r1) > 0 and O.dot(v2, r2) > 0
    v12 = O.vcycle(lev, 2.5 * r1 + r2, p)
    assert np.allclose(v12, 2.5 * v1 + v2, rtol=1e-12, atol=1e-12 * np.abs(v12).max())
    x, hist, st = O.solve(lev, P["b"], 1e-10, params=p)
    assert st == O.OK
