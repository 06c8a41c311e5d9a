"""Pins of the nonsymmetric-operator oracle (oracle/ns.py) against facts that
do not come from it: the symmetric oracle (its own pins) in the symmetric
case, the definition of the directed flux form entry by entry, dense linear
algebra, the piecewise-constant Galerkin product, finite differences and
the divergence-free construction of the synthetic transport."""
import numpy as np
import pytest

from oracle import ns as N
from oracle import tpmg as O
from synthetic import make_ns_problem, make_problem


def _random_directed(nlon, nlat, nz, seed, skew=1.0):
    """Arbitrary nonnegative directed couplings (zero pole and top faces) and
    positive masses: an M-matrix with no structure beyond the form."""
    rng = np.random.default_rng(seed)
    shape = (nz, nlat, nlon)
    h = rng.uniform(0.5, 1.5, shape)
    c = {}
    for name in ("tx", "ty", "tz"):
        base = rng.uniform(0.2, 2.0, shape)
        c[name] = base * rng.uniform(1.0 - 0.5 * skew, 1.0 + 0.5 * skew, shape)
        c[name + "r"] = base * rng.uniform(1.0 - 0.5 * skew, 1.0 + 0.5 * skew, shape)
    for name in ("ty", "tyr"):
        c[name][:, -1, :] = 0.0
    for name in ("tz", "tzr"):
        c[name][-1] = 0.0
    return h, c


def _levels(h, c, params=None, galerkin=False):
    return N.build_hierarchy(h, c["tx"], c["ty"], c["tz"], c["txr"], c["tyr"], c["tzr"],
                             params or O.MGParams(), galerkin=galerkin)


def _dense(lev):
    n = lev.h.size
    A = np.empty((n, n))
    e = np.zeros(n)
    for col in range(n):
        e[col] = 1.0
        A[:, col] = N.apply(lev, e.reshape(lev.shape)).ravel()
        e[col] = 0.0
    return A


def _ns(P):
    return {k: P[k] for k in ("tx", "ty", "tz", "txr", "tyr", "tzr")}


# ----------------------------------------------------------------- the input
def test_transport_is_divergence_free_and_keeps_both_masses():
    P = make_ns_problem(32, 16, 8, 0.2, 5, pe=0.3)
    fx, fy, fz = P["fx"], P["fy"], P["fz"]
    div = fx - np.roll(fx, 1, axis=2)
    div = div + fy
    div[:, 1:, :] -= fy[:, :-1, :]
    div = div + fz
    div[1:] -= fz[:-1]
    assert np.max(np.abs(div)) <= 1e-14 * np.max(np.abs(fx))
    assert np.all(fy[:, -1, :] == 0) and np.all(fz[-1] == 0)
    lev = _levels(P["h"], _ns(P))[0]
    assert np.max(np.abs(N.column_mass(lev) / P["h"] - 1.0)) < 1e-7
    # a real nonsymmetry: the two couplings of a face differ by up to tens of percent
    assert np.max(np.abs(P["tx"] - P["txr"]) / P["tx"]) > 0.1


# ----------------------------------------------------------------- symmetric case
def test_symmetric_case_equals_the_symmetric_oracle():
    P = make_problem(32, 16, 8, 0.2, 5)
    c = {"tx": P["tx"], "ty": P["ty"], "tz": P["tz"],
         "txr": P["tx"], "tyr": P["ty"], "tzr": P["tz"]}
    p = O.MGParams()
    sym = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], p)
    ns = _levels(P["h"], c, p)
    assert len(sym) == len(ns)
    for a, b in zip(sym, ns):
        for x, y in zip(a.coeffs(), (b.tx, b.ty, b.tz, b.h)):
            assert np.array_equal(x, y)
        assert np.array_equal(b.txr, b.tx) and np.array_equal(b.tyr, b.ty)
        assert np.array_equal(N.column_mass(b), b.h)
    u = np.random.default_rng(1).standard_normal(P["h"].shape)
    L0, S0 = ns[0], sym[0]
    assert np.array_equal(N.apply(L0, u), O.apply(S0, u))
    assert np.array_equal(N.column_solve(L0, u), O.column_solve(S0, u))
    w = u.copy()
    O.smooth(S0, P["b"], w, 0.85)
    assert np.array_equal(N.smooth(L0, P["b"], u, 0.85), w)
    z = N.smooth_from_zero(L0, P["b"], 0.85)
    assert np.array_equal(N.presmooth_residual(L0, P["b"], z, 0.85),
                          O.presmooth_residual(S0, P["b"], z, 0.85))
    assert np.array_equal(N.vcycle(ns, P["b"], p), O.vcycle(sym, P["b"], p))


# ----------------------------------------------------------------- the operator
def test_dense_entries_follow_the_directed_flux_form():
    h, c = _random_directed(6, 4, 3, 11)
    lev = _levels(h, c, O.MGParams(levels=1))[0]
    A = _dense(lev)
    nz, nlat, nlon = h.shape
    ix = lambda k, j, i: (k * nlat + j) * nlon + (i % nlon)
    for k in range(nz):
        for j in range(nlat):
            for i in range(nlon):
                cc = ix(k, j, i)
                assert A[cc, ix(k, j, i + 1)] == -c["tx"][k, j, i]
                assert A[ix(k, j, i + 1), cc] == -c["txr"][k, j, i]
                if j + 1 < nlat:
                    assert A[cc, ix(k, j + 1, i)] == -c["ty"][k, j, i]
                    assert A[ix(k, j + 1, i), cc] == -c["tyr"][k, j, i]
                if k + 1 < nz:
                    assert A[cc, ix(k + 1, j, i)] == -c["tz"][k, j, i]
                    assert A[ix(k + 1, j, i), cc] == -c["tzr"][k, j, i]
    # at most 7 entries per row, H 1 = h (row sums), 1' H = h^T (column sums)
    assert np.max(np.count_nonzero(A, axis=1)) <= 7
    assert np.allclose(A.sum(axis=1), h.ravel(), rtol=1e-12, atol=1e-12)
    assert np.allclose(A.sum(axis=0), N.column_mass(lev).ravel(), rtol=1e-12, atol=1e-12)
    # the transposed level is the dense transpose
    assert np.allclose(_dense(N.transpose(lev)), A.T, rtol=0, atol=1e-13)


def test_column_solve_and_sweep_against_dense():
    h, c = _random_directed(6, 4, 5, 12)
    lev = _levels(h, c, O.MGParams(levels=1))[0]
    A = _dense(lev)
    n = h.size
    ncol = h.shape[1] * h.shape[2]
    idx = np.arange(n)
    Hz = np.where((idx[:, None] % ncol) == (idx[None, :] % ncol), A, 0.0)
    rng = np.random.default_rng(3)
    r, b, u = (rng.standard_normal(h.shape) for _ in range(3))
    x = np.linalg.solve(Hz, r.ravel())
    assert np.allclose(N.column_solve(lev, r).ravel(), x, rtol=0, atol=1e-12 * np.abs(x).max())
    om = 0.85
    ref = u.ravel() + om * np.linalg.solve(Hz, b.ravel() - A @ u.ravel())
    assert np.allclose(N.smooth(lev, b, u, om).ravel(), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
    z = N.smooth_from_zero(lev, b, om)
    assert np.allclose(N.presmooth_residual(lev, b, z, om).ravel(), b.ravel() - A @ z.ravel(),
                       rtol=0, atol=1e-12 * np.abs(b).max())


# ----------------------------------------------------------------- coarsening
def _p0(geo_f, geo_c):
    """Piecewise-constant prolongation: each fine cell takes its coarse parent."""
    nz, nlat, nlon = geo_f.shape
    ncj, nci = geo_c.nlat, geo_c.nlon
    P0 = np.zeros((nz * nlat * nlon, nz * ncj * nci))
    for k in range(nz):
        for j in range(nlat):
            for i in range(nlon):
                P0[(k * nlat + j) * nlon + i, (k * ncj + geo_f.row_of[j]) * nci + i // 2] = 1.0
    return P0


def test_unit_factor_coarsening_is_the_galerkin_product():
    h, c = _random_directed(8, 8, 3, 13)
    L = _levels(h, c, O.MGParams(levels=2, alpha_c=0.5), galerkin=True)
    A, Ac = _dense(L[0]), _dense(L[1])
    P0 = _p0(L[0].geo, L[1].geo)
    assert np.allclose(Ac, P0.T @ A @ P0, rtol=0, atol=1e-12 * np.abs(A).max())


def test_default_coarsening_scales_each_face_like_the_symmetric_rule():
    """Each of a face's two couplings is coarsened by the symmetric oracle's
    rule (checked by feeding it the tx/ty/tz of one direction), and the mass
    is the children's sum."""
    h, c = _random_directed(16, 8, 3, 14)
    p = O.MGParams()
    L = _levels(h, c, p)
    for fwd, names in ((True, ("tx", "ty", "tz")), (False, ("txr", "tyr", "tzr"))):
        S = O.build_hierarchy(*(c[k] for k in names), h, p)
        for a, b in zip(S, L):
            got = (b.tx, b.ty, b.tz) if fwd else (b.txr, b.tyr, b.tzr)
            for x, y in zip((a.tx, a.ty, a.tz), got):
                assert np.allclose(x, y, rtol=1e-15, atol=0)
            assert np.allclose(a.h, b.h, rtol=1e-15, atol=0)


def test_transposed_hierarchy_swaps_couplings_and_sums_column_masses():
    P = make_ns_problem(32, 16, 6, 0.2, 6, pe=0.3)
    L = _levels(P["h"], _ns(P))
    T = N.transposed(L)
    for l, (a, b) in enumerate(zip(L, T)):
        assert np.array_equal(b.tx, a.txr) and np.array_equal(b.txr, a.tx)
        assert np.array_equal(b.tyr, a.ty) and np.array_equal(b.tzr, a.tz)
        assert np.all(a.h > 0) and np.all(b.h > 0)
        if l == 0:
            assert np.array_equal(b.h, N.column_mass(a))


# ----------------------------------------------------------------- V-cycle and solves
def test_vcycle_of_the_transpose_is_the_adjoint_on_a_galerkin_hierarchy():
    """With Galerkin coarse operators coarse(H^T) = coarse(H)^T, and the
    V-cycle of H^T (transposed sweeps, R = P^T) is the adjoint of H's."""
    P = make_ns_problem(32, 16, 6, 0.2, 7, pe=0.3)
    L = _levels(P["h"], _ns(P), galerkin=True)
    T = N.transposed(L, galerkin=True)
    p = O.MGParams()
    rng = np.random.default_rng(4)
    for _ in range(3):
        r, s = rng.standard_normal(P["h"].shape), rng.standard_normal(P["h"].shape)
        a = np.vdot(N.vcycle(L, r, p), s)
        b = np.vdot(r, N.vcycle(T, s, p))
        assert abs(a - b) <= 1e-12 * np.linalg.norm(N.vcycle(L, r, p)) * np.linalg.norm(s)
    # and not the adjoint when the coarse operators are rediscretised (R10)
    L2, T2 = _levels(P["h"], _ns(P)), None
    T2 = N.transposed(L2)
    a = np.vdot(N.vcycle(L2, r, p), s)
    b = np.vdot(r, N.vcycle(T2, s, p))
    assert abs(a - b) > 1e-8 * abs(a)


@pytest.mark.parametrize("method", ["stationary", "bicgstab"])
@pytest.mark.parametrize("transpose", [False, True])
def test_solves_match_dense_lu(method, transpose):
    P = make_ns_problem(16, 8, 4, 0.2, 8, pe=0.3)
    L = _levels(P["h"], _ns(P))
    if transpose:
        L = N.transposed(L)
    A = _dense(L[0])
    # the residual floors near 1.4e-11 here (rounding of x times the vertical
    # couplings), so the solve stops at 3e-11 and the solution is compared
    x, hist, st = N.solve(L, P["b"], 3e-11, O.MGParams(method=method, maxit=400))
    assert st == N.OK
    xs = np.linalg.solve(A, P["b"].ravel())
    assert np.linalg.norm(x.ravel() - xs) <= 1e-9 * np.linalg.norm(xs)


def test_nonsymmetric_multigrid_converges_like_the_symmetric_one():
    """The transport makes the operator nonsymmetric by tens of percent per
    face; the V-cycle still reduces the residual at a rate close to the
    symmetric operator's, for H and for H^T."""
    S = make_problem(64, 32, 16, 0.1, 9)
    P = make_ns_problem(64, 32, 16, 0.1, 9, pe=0.3)
    sym = {k: S[k] for k in ("tx", "ty", "tz")}
    sym.update({"txr": S["tx"], "tyr": S["ty"], "tzr": S["tz"]})
    its = {}
    for name, c, b in (("sym", sym, S["b"]), ("ns", _ns(P), P["b"])):
        L = _levels(P["h"] if name == "ns" else S["h"], c)
        for tr in (False, True):
            LL = N.transposed(L) if tr else L
            for m in ("stationary", "bicgstab"):
                x, hist, st = N.solve(LL, b, 1e-10, O.MGParams(method=m, maxit=300))
                assert st == N.OK, (name, tr, m)
                its[(name, tr, m)] = len(hist) - 1
    print(its)
    for tr in (False, True):
        assert its[("ns", tr, "stationary")] <= 1.5 * its[("sym", False, "stationary")] + 2
        assert its[("ns", tr, "bicgstab")] <= 1.5 * its[("sym", False, "bicgstab")] + 2


# ----------------------------------------------------------------- gradient
def test_coefficient_gradient_against_the_linear_dependence_of_h():
    """dL/dtheta_e = -lam^T (dH/dtheta_e) x for every entry e of all seven
    arrays, with dH/dtheta_e x = H_e x where H_e has only theta_e = 1 (H is
    linear in its arrays): built from apply, not from coeff_grad's formula."""
    h, c = _random_directed(4, 4, 3, 15)
    lev = _levels(h, c, O.MGParams(levels=1))[0]
    rng = np.random.default_rng(5)
    x, lam = rng.standard_normal(h.shape), rng.standard_normal(h.shape)
    grads = dict(zip(("h", "tx", "ty", "tz", "txr", "tyr", "tzr"), N.coeff_grad(lev, lam, x)))
    zero = np.zeros_like(h)
    for name in grads:
        for e in range(h.size):
            arrs = {k: zero for k in ("h", "tx", "ty", "tz", "txr", "tyr", "tzr")}
            unit = np.zeros(h.size)
            unit[e] = 1.0
            arrs[name] = unit.reshape(h.shape)
            k, j, i = np.unravel_index(e, h.shape)
            pole = name in ("ty", "tyr") and j == h.shape[1] - 1
            top = name in ("tz", "tzr") and k == h.shape[0] - 1
            He = N.NSLevel(*(arrs[k_] for k_ in ("h", "tx", "ty", "tz", "txr", "tyr", "tzr")),
                           lev.geo)
            want = 0.0 if (pole or top) else -float(np.vdot(lam, N.apply(He, x)))
            assert grads[name].ravel()[e] == pytest.approx(want, rel=1e-12, abs=1e-12)


def test_gradient_of_a_solve_against_central_differences():
    """L(theta) = g^T x(theta), H x = b: the adjoint solve H^T lam = g and
    coeff_grad against central differences of L through dense solves."""
    P = make_ns_problem(8, 4, 3, 0.2, 16, pe=0.3)
    c = _ns(P)
    L = _levels(P["h"], c, O.MGParams(levels=1))
    g = np.random.default_rng(6).standard_normal(P["h"].shape)
    A = _dense(L[0])
    x = np.linalg.solve(A, P["b"].ravel()).reshape(P["h"].shape)
    lam = np.linalg.solve(A.T, g.ravel()).reshape(P["h"].shape)
    grads = dict(zip(("h", "tx", "ty", "tz", "txr", "tyr", "tzr"), N.coeff_grad(L[0], lam, x)))
    arrays = {"h": P["h"], **c}
    rng = np.random.default_rng(7)
    for name, base in arrays.items():
        for _ in range(3):
            e = tuple(rng.integers(0, s) for s in (base.shape[0] - 1, base.shape[1] - 1,
                                                    base.shape[2]))
            step = 1e-6 * base[e]
            vals = []
            for sgn in (1, -1):
                arr = {k: v.copy() for k, v in arrays.items()}
                arr[name][e] += sgn * step
                lv = _levels(arr["h"], {k: arr[k] for k in c}, O.MGParams(levels=1))[0]
                xs = np.linalg.solve(_dense(lv), P["b"].ravel())
                vals.append(float(np.dot(g.ravel(), xs)))
            fd = (vals[0] - vals[1]) / (2 * step)
            assert grads[name][e] == pytest.approx(fd, rel=1e-5, abs=1e-12 * abs(fd) + 1e-30)


# ----------------------------------------------------------------- planted mistakes
def _mut_apply(lev, u):          # west face read from the row's own east couplings
    y = lev.h * u
    y = y + lev.tx * (u - N.east(u))
    y = y + N.west(lev.tx) * (u - N.west(u))
    y = y + lev.ty * (u - N.north(u))
    y = y + N.south(lev.tyr) * (u - N.south(u))
    y = y + lev.tz * (u - N.up(u))
    y = y + N.down(lev.tzr) * (u - N.down(u))
    return y


def _mut_row_sum(lev):           # south coupling dropped from H_z's diagonal
    return lev.h + lev.tx + N.west(lev.txr) + lev.ty


def _mut_transpose(lev):         # row sums kept as the transpose's mass
    return N.NSLevel(lev.h, lev.txr, lev.tyr, lev.tzr, lev.tx, lev.ty, lev.tz, lev.geo)


_real_grad = N.coeff_grad


def _mut_grad(lev, lam, x):      # txr's gradient taken on the wrong row
    g = list(_real_grad(lev, lam, x))
    g[4] = -lam * (N.east(x) - x)
    return tuple(g)


_real_coarsen = N.coarsen


def _mut_coarsen(f, c_geo, sx=0.5, sy=None):  # tyr coarsened from the forward couplings
    c = _real_coarsen(f, c_geo, sx, sy)
    c2 = _real_coarsen(N.NSLevel(f.h, f.tx, f.ty, f.tz, f.txr, f.ty, f.tzr, f.geo), c_geo, sx, sy)
    c.tyr = c2.tyr
    return c


@pytest.mark.parametrize("name,fn,pin", [
    ("apply", _mut_apply, test_dense_entries_follow_the_directed_flux_form),
    ("horizontal_row_sum", _mut_row_sum, test_column_solve_and_sweep_against_dense),
    ("transpose", _mut_transpose, test_dense_entries_follow_the_directed_flux_form),
    ("coeff_grad", _mut_grad, test_coefficient_gradient_against_the_linear_dependence_of_h),
    ("coarsen", _mut_coarsen, test_default_coarsening_scales_each_face_like_the_symmetric_rule),
])
def test_planted_mistakes_are_caught(monkeypatch, name, fn, pin):
    monkeypatch.setattr(N, name, fn)
    with pytest.raises(AssertionError):
        pin()
