"""Pins of the CPU oracle against what the paper and the mathematics fix.

Every check here compares the oracle with something other than itself: exact
geometric totals, exact rational arithmetic, algebraic identities of the
operator and of the multigrid components, a dense LU solve, manufactured
solutions and the paper's own worked numbers.  tests/test_oracle_mutants.py
plants plausible mistakes in a copy of the oracle and checks that these pins
catch them.
"""
from fractions import Fraction

import numpy as np
import pytest

from oracle import tpmg as O
from synthetic import ShellGrid, make_problem


def small(nlon=16, nlat=8, nz=6, sigma=0.1, seed=3):
    return make_problem(nlon, nlat, nz, sigma, seed)


def levels_of(P, **kw):
    p = O.MGParams(**kw)
    return O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], p), p


# ----------------------------------------------------------------- geometry
def test_shell_volume_and_face_areas_are_exact():
    """Input geometry: cell volumes tile the shell; face areas tile spheres,
    cones and meridional planes (closed forms)."""
    g = ShellGrid(48, 24, 7)
    rf = g.r_faces()
    V = g.volumes().sum() * g.nlon
    assert V == pytest.approx(4.0 / 3.0 * np.pi * (rf[-1] ** 3 - rf[0] ** 3), rel=1e-13)
    K = 1.0
    tx, ty, tz, h = g.geometry_coefficients(K)
    rc = g.r_centres()
    # radial faces: area = tz * dist; summed over a sphere r_{k+1} gives 4 pi r^2
    dz = np.diff(rc)
    area_z = tz[:-1] * dz[:, None]
    assert np.allclose(area_z.sum(axis=1) * g.nlon, 4 * np.pi * rf[1:-1] ** 2, rtol=1e-13)
    # lon faces: sum over a meridian half-plane gives pi (r+^2 - r^2) / 2
    cos_c = np.cos(g.lat_centres())
    area_x = tx * (rc[:, None] * cos_c[None, :] * g.dlon)
    assert np.allclose(area_x.sum(axis=1), 0.5 * np.pi * (rf[1:] ** 2 - rf[:-1] ** 2), rtol=1e-13)
    # lat faces: a cone at theta_f has area 2 pi cos(theta_f) (r+^2 - r^2) / 2
    area_y = ty * (rc[:, None] * g.dlat)
    thf = g.lat_faces()[1:-1]
    want = np.pi * np.cos(thf)[None, :] * (rf[1:] ** 2 - rf[:-1] ** 2)[:, None]
    assert np.allclose(area_y[:, :-1] * g.nlon, want, rtol=1e-12)
    assert np.all(ty[:, -1] == 0) and np.all(tz[-1] == 0)


def test_lon_coupling_ratio_is_courant_squared():
    """Section 2.3: horizontal coupling / Helmholtz term ~ nu^2 with nu = 10
    (nu^2 / cos^2(theta) along longitude on the sphere)."""
    P = make_problem(96, 48, 10, 0.0, 1)
    g = P["grid"]
    j = g.nlat // 2
    ratio = P["tx"][:, j, 0] / P["h"][:, j, 0]
    c2 = np.cos(g.lat_centres()[j]) ** 2
    # K = (nu R dlambda)^2 and the lon spacing at radius r_c is r_c cos(theta) dlambda
    want = 100.0 * (g.radius / g.r_centres()) ** 2
    assert np.allclose(ratio * c2, want, rtol=1e-3)


# ----------------------------------------------------------------- operator
def test_operator_kills_constants_exactly():
    """H 1 = h: every flux term T (u_c - u_nb) vanishes for a constant field."""
    P = small()
    lev = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], O.MGParams(levels=1))[0]
    y = O.apply(lev, np.full(lev.shape, 3.0))
    assert np.array_equal(y, 3.0 * P["h"])


def test_operator_symmetric():
    """<H x, y> = <x, H y>: each face couples its two cells with one T."""
    P = small(nlon=32, nlat=16, nz=9)
    lev = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], O.MGParams(levels=1))[0]
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal((2,) + lev.shape)
    a, b = O.dot(O.apply(lev, x), y), O.dot(x, O.apply(lev, y))
    assert abs(a - b) <= 1e-13 * abs(a)


def test_operator_is_spd_m_matrix():
    """Positive Helmholtz term + non-negative couplings: symmetric M-matrix,
    row sums = h > 0, positive definite (dense Cholesky)."""
    P = small(nlon=8, nlat=4, nz=4)
    lev = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], O.MGParams(levels=1))[0]
    A = O.dense_operator(lev)
    assert np.allclose(A, A.T, rtol=0, atol=1e-12 * np.abs(A).max())
    off = A - np.diag(np.diag(A))
    assert np.all(off <= 0) and np.all(np.diag(A) > 0)
    import math
    rows = np.array([math.fsum(row) for row in A])   # exactly rounded row sums
    assert np.all(np.abs(rows - P["h"].ravel()) <= 1e-14 * np.diag(A))
    np.linalg.cholesky(A)
    # sparsity: at most 7 nonzeros per row (7-point stencil)
    assert (np.abs(A) > 0).sum(axis=1).max() <= 7


def _mms(nlon, nlat, nz, K):
    """Manufactured solution u* = Z(r) Y(theta, lambda), Z = cos(pi (r - R)/top)
    (zero normal derivative at surface and top), Y = cos(theta) cos(lambda)
    (a degree-1 spherical harmonic, Laplace-Beltrami eigenvalue -2).  The
    right-hand side is the exact cell integral of f = u* - K Laplacian(u*):
      int f dV = int Y cos(theta) dtheta dlambda
                 * ( -K [r^2 Z']_{r_k}^{r_{k+1}} + 2 K int Z dr + int Z r^2 dr ).
    Returns the volume-weighted relative L2 error of the discrete solution
    against u* at the cell centres."""
    P = make_problem(nlon, nlat, nz, 0.0, 0, K=K)
    g = P["grid"]
    R, Ht = g.radius, g.top
    rf = g.r_faces()
    thf = g.lat_faces()
    lamf = np.arange(nlon + 1) * g.dlon
    a = np.pi / Ht
    Z = lambda r: np.cos(a * (r - R))
    Zp = lambda r: -a * np.sin(a * (r - R))
    r2Zp = rf ** 2 * Zp(rf)
    intZ = (np.sin(a * (rf[1:] - R)) - np.sin(a * (rf[:-1] - R))) / a
    xg, wg = np.polynomial.legendre.leggauss(12)
    mid, half = 0.5 * (rf[1:] + rf[:-1]), 0.5 * (rf[1:] - rf[:-1])
    rr = mid[:, None] + half[:, None] * xg[None, :]
    intZr2 = (half[:, None] * wg[None, :] * Z(rr) * rr ** 2).sum(axis=1)
    radial = -K * np.diff(r2Zp) + 2 * K * intZ + intZr2                 # [nz]
    ang_t = np.diff(thf / 2 + np.sin(2 * thf) / 4)                     # int cos^2
    ang_l = np.diff(np.sin(lamf))                                       # int cos
    b = radial[:, None, None] * ang_t[None, :, None] * ang_l[None, None, :]
    lam = g.lon_centres()[None, None, :]
    th = g.lat_centres()[None, :, None]
    u = Z(g.r_centres())[:, None, None] * np.cos(th) * np.cos(lam)
    lev = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], O.MGParams())
    x, _, st = O.solve(lev, b, 1e-11)
    assert st == O.OK
    e = x - u
    return np.sqrt(np.sum(P["h"] * e * e) / np.sum(P["h"] * u * u))


def test_manufactured_solution_second_order():
    """The flux-form operator approximates (1 - K Laplacian) integrated over
    the cell; its discrete solution converges at second order."""
    K = (10 * 6371e3 * 2 * np.pi / 64) ** 2
    errs = [_mms(n, n // 2, n // 4, K) for n in (32, 64, 128)]
    orders = [np.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) >= 1.9, (errs, orders)


# ----------------------------------------------------------- column solve / Eq. (1)
def _exact_column_solve(diag, off, rhs, exact=False):
    """Gaussian elimination in exact rational arithmetic (sub = super = off);
    exact: return the rationals instead of their rounding."""
    n = len(diag)
    d = list(diag)
    r = [v if isinstance(v, Fraction) else Fraction(float(v)) for v in rhs]
    for k in range(1, n):
        m = off[k - 1] / d[k - 1]
        d[k] -= m * off[k - 1]
        r[k] -= m * r[k - 1]
    x = [Fraction(0)] * n
    x[-1] = r[-1] / d[-1]
    for k in range(n - 2, -1, -1):
        x[k] = (r[k] - off[k] * x[k + 1]) / d[k]
    return x if exact else np.array([float(v) for v in x])


def test_column_solve_matches_exact_rational_solve_of_Hz():
    """H_z (Section 2.1) = the diagonal of H plus its couplings within a
    column.  Its entries, formed exactly from the coefficients, agree with
    the dense H (built by applying the operator to unit vectors), and the
    oracle's column solve matches an exact rational solve of it."""
    P = small(nlon=8, nlat=4, nz=12, sigma=0.2)
    lev = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], O.MGParams(levels=1))[0]
    A = O.dense_operator(lev)
    rng = np.random.default_rng(1)
    r = rng.uniform(-1, 1, lev.shape)
    x = O.column_solve(lev, r)
    nz, nlat, nlon = lev.shape
    tx, ty, tz, h = (P[k] for k in ("tx", "ty", "tz", "h"))
    F = lambda v: Fraction(float(v))
    for (j, i) in [(0, 0), (1, 5), (3, 7), (2, 2)]:
        idx = [(k * nlat + j) * nlon + i for k in range(nz)]
        Hz = A[np.ix_(idx, idx)]
        diag = []
        for k in range(nz):
            d = F(h[k, j, i]) + F(tx[k, j, i]) + F(tx[k, j, i - 1]) + F(ty[k, j, i])
            d += F(ty[k, j - 1, i]) if j > 0 else 0
            d += F(tz[k, j, i]) + (F(tz[k - 1, j, i]) if k > 0 else 0)
            diag.append(d)
        off = [-F(tz[k, j, i]) for k in range(nz - 1)]
        assert np.allclose(np.diag(Hz), [float(d) for d in diag], rtol=4e-16, atol=0)
        assert np.array_equal(np.diag(Hz, 1), [float(o) for o in off])
        xe = _exact_column_solve(diag, off, r[:, j, i])
        assert np.max(np.abs(x[:, j, i] - xe)) <= 1e-13 * np.max(np.abs(xe))


def _exact_residual_form_sweep(P, b, u, omega):
    """Eq. (1) as printed (with the convergent sign), in exact rational
    arithmetic: u + omega H_z^{-1} (b - H u), with H from the definition."""
    tx, ty, tz, h = (P[k] for k in ("tx", "ty", "tz", "h"))
    nz, nlat, nlon = h.shape
    F = lambda v: Fraction(float(v))
    U = {(k, j, i): F(u[k, j, i]) for k in range(nz) for j in range(nlat) for i in range(nlon)}
    out = np.empty_like(u)
    for j in range(nlat):
        for i in range(nlon):
            r, diag, off = [], [], []
            for k in range(nz):
                c = U[k, j, i]
                faces = [(F(tx[k, j, i]), U[k, j, (i + 1) % nlon]),
                         (F(tx[k, j, i - 1]), U[k, j, (i - 1) % nlon])]
                if j + 1 < nlat:
                    faces.append((F(ty[k, j, i]), U[k, j + 1, i]))
                if j > 0:
                    faces.append((F(ty[k, j - 1, i]), U[k, j - 1, i]))
                if k + 1 < nz:
                    faces.append((F(tz[k, j, i]), U[k + 1, j, i]))
                if k > 0:
                    faces.append((F(tz[k - 1, j, i]), U[k - 1, j, i]))
                hu = F(h[k, j, i]) * c + sum(t * (c - un) for t, un in faces)
                r.append(F(b[k, j, i]) - hu)
                diag.append(F(h[k, j, i]) + sum(t for t, _ in faces))
                if k + 1 < nz:
                    off.append(-F(tz[k, j, i]))
            # exact tridiagonal solve
            d, rr = list(diag), list(r)
            for k in range(1, nz):
                m = off[k - 1] / d[k - 1]
                d[k] -= m * off[k - 1]
                rr[k] -= m * rr[k - 1]
            x = [Fraction(0)] * nz
            x[-1] = rr[-1] / d[-1]
            for k in range(nz - 2, -1, -1):
                x[k] = (rr[k] - off[k] * x[k + 1]) / d[k]
            for k in range(nz):
                out[k, j, i] = float(U[k, j, i] + F(omega) * x[k])
    return out


def _exact_presmooth_residual(P, b, omega):
    """b - H u for u = omega H_z^{-1} b, all in exact rational arithmetic,
    H and H_z written out from the coefficients."""
    tx, ty, tz, h = (P[k] for k in ("tx", "ty", "tz", "h"))
    nz, nlat, nlon = h.shape
    F = lambda v: Fraction(float(v))
    U = {}
    for j in range(nlat):
        for i in range(nlon):
            diag, off = [], []
            for k in range(nz):
                d = F(h[k, j, i]) + F(tx[k, j, i]) + F(tx[k, j, i - 1])
                d += F(ty[k, j, i]) if j + 1 < nlat else 0
                d += F(ty[k, j - 1, i]) if j > 0 else 0
                d += F(tz[k, j, i]) if k + 1 < nz else 0
                d += F(tz[k - 1, j, i]) if k > 0 else 0
                diag.append(d)
                if k + 1 < nz:
                    off.append(-F(tz[k, j, i]))
            x = _exact_column_solve(diag, off, [F(b[k, j, i]) for k in range(nz)], exact=True)
            for k in range(nz):
                U[k, j, i] = F(omega) * x[k]
    r = np.empty(h.shape)
    for k in range(nz):
        for j in range(nlat):
            for i in range(nlon):
                c = U[k, j, i]
                faces = [(F(tx[k, j, i]), U[k, j, (i + 1) % nlon]),
                         (F(tx[k, j, i - 1]), U[k, j, (i - 1) % nlon])]
                if j + 1 < nlat:
                    faces.append((F(ty[k, j, i]), U[k, j + 1, i]))
                if j > 0:
                    faces.append((F(ty[k, j - 1, i]), U[k, j - 1, i]))
                if k + 1 < nz:
                    faces.append((F(tz[k, j, i]), U[k + 1, j, i]))
                if k > 0:
                    faces.append((F(tz[k - 1, j, i]), U[k - 1, j, i]))
                hu = F(h[k, j, i]) * c + sum(t * (c - un) for t, un in faces)
                r[k, j, i] = float(F(b[k, j, i]) - hu)
    return r


def test_presmooth_residual_is_the_exact_residual_of_the_sweep():
    """After one sweep from zero, u = omega H_z^{-1} b, the V-cycle takes the
    residual as (1 - omega) b plus the horizontal couplings of u: against b -
    H u of the exact sweep in rational arithmetic it agrees to 1e-13, closer
    than the flux form b - H u of the rounded sweep, which carries the
    rounding of the column solve times the vertical couplings."""
    P = small(nlon=8, nlat=4, nz=6, sigma=0.2)
    lev = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], O.MGParams(levels=1))[0]
    b = P["b"]
    u = np.zeros(lev.shape)
    O.smooth(lev, b, u, 0.85)
    want = _exact_presmooth_residual(P, b, 0.85)
    got = O.presmooth_residual(lev, b, u, 0.85)
    scale = np.max(np.abs(want))
    assert np.max(np.abs(got - want)) <= 1e-13 * scale
    flux = O.residual(lev, b, u)
    assert np.max(np.abs(got - want)) <= np.max(np.abs(flux - want))


def test_smoother_is_eq1_with_convergent_sign():
    """One sweep equals Eq. (1) with the '+' sign, u + omega H_z^{-1}(b - H u),
    evaluated exactly in rational arithmetic (the oracle evaluates the same
    iteration as (1 - omega) u + omega H_z^{-1}(b - dH u)); repeated sweeps
    reduce the error (the printed '-' sign diverges)."""
    P = small(nlon=8, nlat=4, nz=6, sigma=0.2)
    lev = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], O.MGParams(levels=1))[0]
    rng = np.random.default_rng(2)
    u = rng.standard_normal(lev.shape)
    b = P["b"]
    u1 = u.copy()
    O.smooth(lev, b, u1, 0.8)
    want = _exact_residual_form_sweep(P, b, u, 0.8)
    assert np.max(np.abs(u1 - want)) <= 1e-14 * np.max(np.abs(want))
    xs, _ = _dense_solve(P, b)
    e0 = np.linalg.norm(u - xs)
    for _ in range(30):
        O.smooth(lev, b, u, 0.8)
    assert np.linalg.norm(u - xs) < 0.5 * e0


# ----------------------------------------------------------------- hierarchy
def test_row_maps_worked_example_64x32():
    """Conditional semi-coarsening (Section 2.2) worked by hand for 64x32,
    alpha_c = 1/2: level 1 merges the 5 equatorial pairs of each hemisphere
    (centres up to 50.6 deg; the next pair at 61.9 deg has cos < 1/2), level
    2 merges 4 pairs, level 3 merges 3 pairs."""
    P = make_problem(64, 32, 4, 0.1, 0)
    lev, _ = levels_of(P, levels=4, alpha_c=0.5)
    assert [(l.nlon, l.nlat) for l in lev] == [(64, 32), (32, 22), (16, 14), (8, 8)]
    # level 1: rows 16..25 merged in pairs, 26..31 single
    r = lev[0].row_of
    assert list(r[16:26]) == [11, 11, 12, 12, 13, 13, 14, 14, 15, 15]
    assert list(r[26:32]) == [16, 17, 18, 19, 20, 21]
    # mirror symmetry
    assert np.allclose(lev[1].south, -lev[1].north[::-1])


def test_row_maps_properties():
    """Longitude always halves; merged rows form one band around the equator
    in which every merged cell keeps alpha >= alpha_c."""
    P = make_problem(256, 192, 2, 0.1, 0)
    lev, p = levels_of(P)
    for f, c in zip(lev[:-1], lev[1:]):
        assert c.nlon == f.nlon // 2
        cnt = np.bincount(f.row_of)
        assert set(cnt) <= {1, 2}
        merged = np.nonzero(cnt == 2)[0]
        if len(merged):
            assert np.all(np.diff(merged) == 1)          # one contiguous band
            assert merged[0] + merged[-1] == c.nlat - 1  # centred on the equator
            cc = c.centres[merged]
            dth = (c.north - c.south)[merged]
            alpha = np.cos(cc) * (2 * np.pi / c.nlon) / dth
            assert np.all(alpha >= p.alpha_c)


@pytest.mark.parametrize("alpha_c", [0.3, 0.5, 0.6, 0.9])
def test_restriction_gathers_at_most_four_fine_rows(alpha_c):
    """R = P^T in latitude: a coarse row collects its one or two children
    and, from each neighbouring merged pair, only the child nearer to it (a
    single child sits at its parent's centre and interpolates nowhere) --
    at most 4 fine rows, the bound the GPU restriction is built for."""
    P = make_problem(256, 192, 2, 0.1, 0)
    lev, _ = levels_of(P, alpha_c=alpha_c)
    for f in lev[:-1]:
        j0, w0, j1, w1 = f.links()
        gathered = np.bincount(j0, minlength=f.nlat_c) + np.bincount(j1[j1 >= 0],
                                                                     minlength=f.nlat_c)
        assert gathered.max() <= 4
        single = np.bincount(f.row_of, minlength=f.nlat_c)[f.row_of] == 1
        assert np.all(j1[single] == -1)      # a lone child interpolates nowhere


def _dense(lev):
    n = lev.size
    A = np.empty((n, n))
    e = np.zeros(n)
    for c in range(n):
        e[c] = 1.0
        A[:, c] = O.apply(lev, e.reshape(lev.shape)).ravel()
        e[c] = 0.0
    return A


def _dense_column_blocks(lev):
    """H_z written out: per column the tridiagonal with diagonal h + the six
    face couplings and off-diagonals -t_z (Eq. (1)'s split)."""
    nz, nlat, nlon = lev.shape
    idx = np.arange(lev.size).reshape(lev.shape)
    Hz = np.zeros((lev.size, lev.size))
    for k in range(nz):
        for j in range(nlat):
            for i in range(nlon):
                c = idx[k, j, i]
                d = lev.h[k, j, i] + lev.tx[k, j, i] + lev.tx[k, j, (i - 1) % nlon]
                if j + 1 < nlat:
                    d += lev.ty[k, j, i]
                if j > 0:
                    d += lev.ty[k, j - 1, i]
                if k + 1 < nz:
                    d += lev.tz[k, j, i]
                    Hz[c, idx[k + 1, j, i]] = -lev.tz[k, j, i]
                if k > 0:
                    d += lev.tz[k - 1, j, i]
                    Hz[c, idx[k - 1, j, i]] = -lev.tz[k - 1, j, i]
                Hz[c, c] = d
    return Hz


def test_coarse_pcg_first_step_and_finite_termination():
    """The PCG form of the coarsest-grid iteration: its first iterate is the
    exact line search along z = H_z^{-1} b (H_z assembled by hand), the
    H-norm error falls monotonically, and after n iterations on n unknowns
    it reaches the dense solution (finite termination of CG)."""
    P = small(nlon=8, nlat=4, nz=3, sigma=0.2, seed=5)
    lev = levels_of(P, levels=1)[0][0]
    A = _dense(lev)
    b = np.random.default_rng(8).standard_normal(lev.shape)
    z = np.linalg.solve(_dense_column_blocks(lev), b.ravel())
    x1 = (b.ravel() @ z) / (z @ A @ z) * z
    # cond(H_z) ~ 3e4 here: the dense solve itself is good to ~1e-12
    assert np.abs(O.coarse_pcg(lev, b, 1).ravel() - x1).max() <= 1e-10 * np.abs(x1).max()
    xs = np.linalg.solve(A, b.ravel())
    errs = []
    for it in (1, 2, 4, 8, 16):
        e = O.coarse_pcg(lev, b, it).ravel() - xs
        errs.append(e @ A @ e)
    assert all(a > b_ for a, b_ in zip(errs, errs[1:]))
    x = O.coarse_pcg(lev, b, lev.size).ravel()
    assert np.linalg.norm(x - xs) <= 1e-9 * np.linalg.norm(xs)
    assert np.array_equal(O.coarse_pcg(lev, np.zeros(lev.shape), 5), np.zeros(lev.shape))


def test_coarse_pcg_in_the_vcycle():
    """coarse_method = "pcg" replaces the coarsest level's sweeps: a V-cycle
    over one level is the PCG itself, and with enough iterations a two-level
    cycle's coarse correction solves the coarse system exactly."""
    P = small(nlon=16, nlat=8, nz=3, sigma=0.1, seed=6)
    lev, p = levels_of(P, levels=2, coarse_method="pcg", coarse_iters=200)
    b = np.random.default_rng(9).standard_normal(lev[1].shape)
    xs = np.linalg.solve(_dense(lev[1]), b.ravel())
    got = O.vcycle(lev, b, p, l=1).ravel()
    assert np.linalg.norm(got - xs) <= 1e-9 * np.linalg.norm(xs)


def test_coarse_operator_conserves_volume_and_stays_spd():
    P = small(nlon=16, nlat=8, nz=3)
    lev, _ = levels_of(P, levels=3)
    for l in lev:
        assert l.h.sum() == pytest.approx(P["h"].sum(), rel=1e-13)
        A = O.dense_operator(l)
        assert np.allclose(A, A.T, atol=1e-12 * np.abs(A).max())
        np.linalg.cholesky(A)


def test_transfers_adjoint_and_exact_for_linear_fields():
    """R = P^T; P preserves constants and, away from the poles, fields
    linear in latitude and in longitude (bilinear interpolation)."""
    P = make_problem(64, 32, 3, 0.1, 0)
    lev, _ = levels_of(P, levels=3)
    rng = np.random.default_rng(4)
    for f, c in zip(lev[:-1], lev[1:]):
        r = rng.standard_normal(f.shape)
        e = rng.standard_normal(c.shape)
        u = np.zeros(f.shape)
        O.prolong_add(f, e, u)
        a, b = O.dot(O.restrict(f, r), e), O.dot(r, u)
        assert abs(a - b) <= 1e-13 * abs(a)
        one = np.zeros(f.shape)
        O.prolong_add(f, np.ones(c.shape), one)
        assert np.allclose(one, 1.0, rtol=0, atol=1e-15)
        th = np.zeros(f.shape)
        O.prolong_add(f, np.broadcast_to(c.centres[None, :, None], c.shape).copy(), th)
        inner = (f.centres > c.centres[0]) & (f.centres < c.centres[-1])
        want = np.broadcast_to(f.centres[None, :, None], f.shape)
        assert np.allclose(th[:, inner, :], want[:, inner, :], atol=1e-14)
        lam_c = np.cos((np.arange(c.nlon) + 0.5) * 2 * np.pi / c.nlon)
        lam_f = np.cos((np.arange(f.nlon) + 0.5) * 2 * np.pi / f.nlon)
        ul = np.zeros(f.shape)
        O.prolong_add(f, np.broadcast_to(lam_c[None, None, :], c.shape).copy(), ul)
        # linear interpolation of cos: error <= (dlam_c/2)^2 * 3/16 ... bound by the spacing
        assert np.max(np.abs(ul - lam_f[None, None, :])) <= (2 * np.pi / c.nlon) ** 2 / 4


# ----------------------------------------------------------------- V-cycle / solve
def test_vcycle_symmetric_positive_linear():
    """The V-cycle is a fixed symmetric positive-definite linear operator
    (what conjugate gradients and the adjoint solve need)."""
    P = make_problem(32, 16, 8, 0.1, 5)
    lev, p = levels_of(P)
    rng = np.random.default_rng(5)
    r1, r2 = rng.standard_normal((2,) + lev[0].shape)
    v1, v2 = O.vcycle(lev, r1, p), O.vcycle(lev, r2, p)
    a, b = O.dot(v1, r2), O.dot(r1, v2)
    assert abs(a - b) <= 1e-12 * abs(a)
    assert O.dot(v1, r1) > 0 and O.dot(v2, r2) > 0
    v12 = O.vcycle(lev, 2.5 * r1 + r2, p)
    assert np.allclose(v12, 2.5 * v1 + v2, rtol=1e-12, atol=1e-12 * np.abs(v12).max())


def _assemble_offdiag_and_rowsums(P):
    """Dense off-diagonal part (-T for each face) and row sums (h) of H."""
    tx, ty, tz, h = (P[k] for k in ("tx", "ty", "tz", "h"))
    nz, nlat, nlon = h.shape
    n = h.size
    A = np.zeros((n, n))
    idx = lambda k, j, i: (k * nlat + j) * nlon + i
    for k in range(nz):
        for j in range(nlat):
            for i in range(nlon):
                c = idx(k, j, i)
                for nb, t in ((idx(k, j, (i + 1) % nlon), tx[k, j, i]),
                              (idx(k, j + 1, i) if j + 1 < nlat else -1, ty[k, j, i]),
                              (idx(k + 1, j, i) if k + 1 < nz else -1, tz[k, j, i])):
                    if nb >= 0 and nb != c:
                        A[c, nb] -= t
                        A[nb, c] -= t
    return A, h.ravel().copy()


def _dense_solve(P, b):
    A_off, s = _assemble_offdiag_and_rowsums(P)
    n = len(s)
    A = A_off.copy()
    s = s.copy()
    rhs = b.ravel().astype(np.float64).copy()
    d = np.zeros(n)
    Urows = []
    for k in range(n):
        offrow = A[k, k + 1:].copy()
        d[k] = s[k] - offrow.sum()
        col = A[k + 1:, k].copy()
        m = col / d[k]
        A[k + 1:, k + 1:] -= np.outer(m, offrow)
        np.fill_diagonal(A[k + 1:, k + 1:], 0.0)
        s[k + 1:] -= m * s[k]
        rhs[k + 1:] -= m * rhs[k]
        Urows.append(offrow)
    x = np.zeros(n)
    for k in range(n - 1, -1, -1):
        x[k] = (rhs[k] - Urows[k] @ x[k + 1:]) / d[k]
    return x.reshape(b.shape), A_off


@pytest.mark.parametrize("shape", [(8, 4, 4), (16, 8, 4), (16, 8, 6)])
def test_solve_matches_dense_lu(shape):
    """Multigrid solve (40 iterations, past the FP64 floor) vs a dense LU
    solve of H (tiny grids), the LU carried out in the row-sum form that
    keeps full relative accuracy.  On these grids the residual of even the
    correctly rounded solution is ~1e-11 relative (rounding of x times the
    vertical couplings), so the pin is on the solution, to 1e-12."""
    P = make_problem(*shape, 0.1, 11)
    lev, p = levels_of(P)
    x, hist, st = O.solve(lev, P["b"], 0.0, params=p, maxit=40)
    assert hist[-1] < 1e-10
    xd, A_off = _dense_solve(P, P["b"])
    A = O.dense_operator(lev[0])
    off = A - np.diag(np.diag(A))
    assert np.array_equal(off, A_off)          # the oracle's operator is this matrix
    assert np.linalg.norm(x - xd) <= 1e-12 * np.linalg.norm(xd)


def test_stationary_and_cg_agree():
    P = make_problem(64, 32, 16, 0.1, 1000)
    lev, p = levels_of(P, method="stationary")
    xs, _, st1 = O.solve(lev, P["b"], 1e-11, params=p)
    xc, _, st2 = O.solve(lev, P["b"], 1e-11)
    assert st1 == st2 == O.OK
    assert np.linalg.norm(xs - xc) <= 1e-9 * np.linalg.norm(xc)


def test_stationary_residual_decreases_monotonically():
    """Section 2.4: multigrid converges monotonically."""
    P = make_problem(64, 32, 16, 0.1, 1000)
    lev, p = levels_of(P, method="stationary")
    _, hist, st = O.solve(lev, P["b"], 1e-10, params=p)
    assert st == O.OK
    assert all(b < a for a, b in zip(hist, hist[1:]))


def test_mixed_precision_reaches_fp64_solution():
    P = make_problem(64, 32, 16, 0.1, 1000)
    lev, p = levels_of(P)
    xr, _, _ = O.solve(lev, P["b"], 1e-13, params=p)
    xm, hist, st = O.solve_mixed(lev, P["b"], 1e-10, params=p)
    assert st == O.OK and hist[-1] <= 1e-10
    assert np.linalg.norm(xm - xr) <= 1e-9 * np.linalg.norm(xr)
    assert len(hist) <= 8


# ----------------------------------------------------------------- gradient
def test_gradient_matches_dense_lu_and_finite_differences():
    """Differentiable solve: dL/db = lambda, dL/dh = -lambda x and
    dL/dT = -(lambda_1 - lambda_2)(x_1 - x_2) for L = 0.5 ||W x||^2, against
    a dense-LU reference gradient and central differences (step 1e-6 on
    unit directions); every dense solve in the row-sum form."""
    P = make_problem(8, 4, 4, 0.1, 21)
    rng = np.random.default_rng(22)
    W = rng.uniform(0, 1, P["h"].shape)
    lev, p = levels_of(P)
    x, g = O.solve_with_grad(lev, P["b"], lambda x: W * W * x, tol=1e-11, params=p)
    xd, _ = _dense_solve(P, P["b"])
    lam, _ = _dense_solve(P, W * W * xd)
    assert np.linalg.norm(g["b"] - lam) <= 1e-10 * np.linalg.norm(lam)
    assert np.linalg.norm(g["h"] + lam * xd) <= 1e-10 * np.linalg.norm(lam * xd)

    def loss(**over):
        Q = dict(P)
        Q.update(over)
        xx, _ = _dense_solve(Q, Q["b"])
        return 0.5 * np.sum((W * xx) ** 2)

    eps = 1e-6
    for _ in range(4):
        d = rng.standard_normal(P["h"].shape)
        d /= np.linalg.norm(d)
        fd_b = (loss(b=P["b"] + eps * d) - loss(b=P["b"] - eps * d)) / (2 * eps)
        assert abs(fd_b - np.sum(g["b"] * d)) <= 1e-6 * np.linalg.norm(g["b"])
        fd_h = (loss(h=P["h"] * (1 + eps * d)) - loss(h=P["h"] * (1 - eps * d))) / (2 * eps)
        an_h = np.sum(g["h"] * P["h"] * d)
        assert abs(fd_h - an_h) <= 1e-6 * np.linalg.norm(g["h"] * P["h"])
        # face gradients are ~1e-4 of L's scale: a 1e-4 step keeps FP64
        # rounding of L below the tolerance (truncation ~1e-8 relative)
        for key in ("tx", "ty"):
            et = 1e-4
            fd_t = (loss(**{key: P[key] * (1 + et * d)}) -
                    loss(**{key: P[key] * (1 - et * d)})) / (2 * et)
            an_t = np.sum(g[key] * P[key] * d)
            assert abs(fd_t - an_t) <= 1e-6 * np.linalg.norm(g[key] * P[key]), key
        # dL along tz is ~1e-7 of L (the columns are nearly rigid), below
        # what a 1e-6 step resolves in FP64 (rounding noise ~1e-3 relative):
        # step 1e-3, whose O(step^2) truncation is ~1e-5 relative
        e = 1e-3
        fd_t = (loss(tz=P["tz"] * (1 + e * d)) - loss(tz=P["tz"] * (1 - e * d))) / (2 * e)
        an_t = np.sum(g["tz"] * P["tz"] * d)
        assert abs(fd_t - an_t) <= 1e-4 * abs(an_t)
