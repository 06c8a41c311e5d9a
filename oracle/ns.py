"""CPU oracle of the nonsymmetric form of the operator (a generalisation the
paper motivates but does not define: Section 1 names BiCGStab as the solver
of the operational, nonsymmetric Helmholtz problem).

TEST INFRASTRUCTURE ONLY: imported by tests/ and by the package's smoke
check.  The CUDA library never imports it.  Plain numpy (float64), vectorised
over columns; the geometry of the hierarchy (row maps, prolongation weights,
Section 2.2) and the transfers come from the symmetric oracle, which is
pinned on its own.

Operator (directed flux form).  Every face carries two couplings, one per
row that it enters:
  tx[c]: row c's coupling to its east neighbour E   txr[c]: row E's coupling to c
  ty[c]: row c's coupling to its north neighbour N  tyr[c]: row N's coupling to c
  tz[c]: row c's coupling to the layer above U      tzr[c]: row U's coupling to c
and h is the row sum ("mass"):
  (H u)_c = h_c u_c + tx[c](u_c - u_E) + txr[W](u_c - u_W) + ty[c](u_c - u_N)
            + tyr[S](u_c - u_S) + tz[c](u_c - u_U) + tzr[D](u_c - u_D)
with W, S, D the west, south and lower neighbours (whose face arrays hold
the coupling back to c).  Pole, surface and top faces carry zero couplings.
txr = tx, tyr = ty, tzr = tz gives the symmetric operator of Section 2.

Transpose.  H^T has the same form with the two couplings of every face
swapped and the column sums as its mass:
  h^T_c = h_c + sum over the six faces of (row coupling - column coupling).

Smoother (Eq. (1) with H_z the column tridiagonal of the directed operator),
coarsening (R10 applied to both couplings of a face, masses summed), the
hierarchy of H^T (the same rule applied to H^T), V-cycle, stationary and
BiCGStab solves and the coefficient gradient follow.  No function here has a
printed counterpart in the paper; the pins are mathematical (tests/test_oracle_ns.py): the symmetric case
against the symmetric oracle, the dense operator and its transpose, dense
LU, piecewise-constant Galerkin products (and the V-cycle's adjointness on
such a hierarchy), finite differences.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import tpmg as O

OK, NOT_CONVERGED, DIVERGED = 0, 4, 5


@dataclass
class NSLevel:
    h: np.ndarray
    tx: np.ndarray
    ty: np.ndarray
    tz: np.ndarray
    txr: np.ndarray
    tyr: np.ndarray
    tzr: np.ndarray
    geo: O.Level      # shape, row geometry and links to the next level

    @property
    def shape(self):
        return self.h.shape

    def arrays(self):
        return self.h, self.tx, self.ty, self.tz, self.txr, self.tyr, self.tzr


# --------------------------------------------------------------- neighbour shifts
def east(a):
    return np.roll(a, -1, axis=2)


def west(a):
    return np.roll(a, 1, axis=2)


def north(a):
    out = np.zeros_like(a)
    out[:, :-1] = a[:, 1:]
    return out


def south(a):
    out = np.zeros_like(a)
    out[:, 1:] = a[:, :-1]
    return out


def up(a):
    out = np.zeros_like(a)
    out[:-1] = a[1:]
    return out


def down(a):
    out = np.zeros_like(a)
    out[1:] = a[:-1]
    return out


# --------------------------------------------------------------- operator
def apply(lev: NSLevel, u):
    """y = H u in the directed flux form (terms added in the order written in
    the module docstring)."""
    y = lev.h * u
    y = y + lev.tx * (u - east(u))
    y = y + west(lev.txr) * (u - west(u))
    y = y + lev.ty * (u - north(u))
    y = y + south(lev.tyr) * (u - south(u))
    y = y + lev.tz * (u - up(u))
    y = y + down(lev.tzr) * (u - down(u))
    return y


def residual(lev: NSLevel, b, u):
    return b - apply(lev, u)


def column_mass(lev: NSLevel):
    """h^T: the column sums of H, h plus (row - column) coupling of each of
    the six faces; zero differences where the two couplings agree."""
    d = lev.h + (lev.tx - lev.txr)
    d = d + (west(lev.txr) - west(lev.tx))
    d = d + (lev.ty - lev.tyr)
    d = d + (south(lev.tyr) - south(lev.ty))
    d = d + (lev.tz - lev.tzr)
    d = d + (down(lev.tzr) - down(lev.tz))
    return d


def transpose(lev: NSLevel) -> NSLevel:
    """H^T: the couplings of every face swapped, the column sums as mass."""
    return NSLevel(column_mass(lev), lev.txr, lev.tyr, lev.tzr, lev.tx, lev.ty, lev.tz, lev.geo)


# --------------------------------------------------------------- smoother (Eq. (1))
def horizontal_row_sum(lev: NSLevel):
    """s = h + the row's four horizontal couplings: the diagonal of H_z less
    its two vertical couplings (Section 2.1's split H = H_z + dH)."""
    return lev.h + lev.tx + west(lev.txr) + lev.ty + south(lev.tyr)


def column_solve(lev: NSLevel, r):
    """x = H_z^{-1} r for every column.  Row k of H_z: -l_k x_{k-1} + (s_k +
    l_k + u_k) x_k - u_k x_{k+1}, with u_k = tz[k] (coupling to the layer
    above) and l_k = tzr[k-1] (coupling to the layer below).  Gaussian
    elimination in the row-sum form: q_0 = s_0, p_k = q_k + u_k, q_k = s_k +
    l_k q_{k-1} / p_{k-1}; forward y_k = (r_k + l_k y_{k-1}) / p_k; backward
    x_k = x_{k+1} + (y_k - (q_k / p_k) x_{k+1})."""
    s = horizontal_row_sum(lev)
    lo = down(lev.tzr)
    nz = r.shape[0]
    q = np.empty_like(r)
    p = np.empty_like(r)
    y = np.empty_like(r)
    for k in range(nz):
        if k == 0:
            q[0] = s[0]
        else:
            q[k] = s[k] + lo[k] * q[k - 1] / p[k - 1]
        p[k] = q[k] + lev.tz[k]
        y[k] = (r[k] + lo[k] * y[k - 1]) / p[k] if k > 0 else r[0] / p[0]
    x = np.empty_like(r)
    x[nz - 1] = y[nz - 1]
    for k in range(nz - 2, -1, -1):
        x[k] = x[k + 1] + (y[k] - (q[k] / p[k]) * x[k + 1])
    return x


def horizontal_rhs(lev: NSLevel, b, u):
    """b - dH u = b plus the row's four horizontal couplings times u."""
    v = b + lev.tx * east(u)
    v = v + west(lev.txr) * west(u)
    v = v + lev.ty * north(u)
    v = v + south(lev.tyr) * south(u)
    return v


def smooth(lev: NSLevel, b, u, omega: float):
    """One sweep of Eq. (1), u <- (1 - omega) u + omega H_z^{-1}(b - dH u);
    returns the new u (every column reads the old one)."""
    x = column_solve(lev, horizontal_rhs(lev, b, u))
    return (1.0 - omega) * u + omega * x


def smooth_from_zero(lev: NSLevel, b, omega: float):
    return omega * column_solve(lev, b)


def presmooth_residual(lev: NSLevel, b, u, omega: float):
    """b - H u for u = omega H_z^{-1} b: H_z u = omega b leaves (1 - omega) b
    plus the four horizontal couplings of u."""
    v = (1.0 - omega) * b + lev.tx * east(u)
    v = v + west(lev.txr) * west(u)
    v = v + lev.ty * north(u)
    v = v + south(lev.tyr) * south(u)
    return v


# --------------------------------------------------------------- hierarchy
def lat_face_ratios(f: O.Level, c: O.Level):
    """sy[J]: fine centre distance across coarse row J's north face over the
    coarse centre distance (R10's rediscretisation of a latitude face);
    zero on the last coarse row."""
    fc, cc = f.centres, c.centres
    sy = np.zeros(c.nlat)
    for J in range(c.nlat - 1):
        t = f.top_row[J]
        sy[J] = (fc[t + 1] - fc[t]) / (cc[J + 1] - cc[J])
    return sy


def coarsen(f: NSLevel, c_geo: O.Level, sx: float = 0.5, sy=None) -> NSLevel:
    """Coarse operator of the next level (R10 applied to each coupling of a
    face).  A coarse cell is 2 longitudes x its 1 or 2 fine rows of the same
    layer:
      h, tz, tzr: sums over the children (the vertical is never coarsened)
      tx, txr:    sx times the sums over the fine faces forming the coarse
                  east face
      ty, tyr:    sy[J] times the sums over the top child row's north faces
                  (zero on the last coarse row).
    The mass stays the children's sum, so every coarse operator keeps
    positive row sums (an M-matrix like the fine one).  Equal couplings give
    the symmetric rule; sx = sy = 1 gives the Galerkin product P0^T H P0 of
    piecewise-constant prolongation (for which coarse(H^T) = coarse(H)^T)."""
    g = f.geo
    nz, nlat, nlon = f.shape
    ncj, nci = c_geo.nlat, nlon // 2
    if sy is None:
        sy = lat_face_ratios(g, c_geo)
    sy = np.asarray(sy, dtype=np.float64)
    out = {k: np.zeros((nz, ncj, nci)) for k in ("h", "tx", "ty", "tz", "txr", "tyr", "tzr")}
    row_of, top = g.row_of, g.top_row
    for j in range(nlat):
        J = int(row_of[j])
        for name in ("h", "tz", "tzr"):
            a = getattr(f, name)
            out[name][:, J, :] += a[:, j, 0::2]
            out[name][:, J, :] += a[:, j, 1::2]
        out["tx"][:, J, :] += f.tx[:, j, 1::2]
        out["txr"][:, J, :] += f.txr[:, j, 1::2]
        if j == top[J]:
            for name in ("ty", "tyr"):
                a = getattr(f, name)
                out[name][:, J, :] += a[:, j, 0::2]
                out[name][:, J, :] += a[:, j, 1::2]
    out["tx"] *= sx
    out["txr"] *= sx
    out["ty"] *= sy[:, None]
    out["tyr"] *= sy[:, None]
    out["ty"][:, ncj - 1, :] = 0.0
    out["tyr"][:, ncj - 1, :] = 0.0
    return NSLevel(out["h"], out["tx"], out["ty"], out["tz"], out["txr"], out["tyr"], out["tzr"],
                   c_geo)


def build_hierarchy(h, tx, ty, tz, txr, tyr, tzr, params: O.MGParams | None = None,
                    galerkin: bool = False):
    """Levels 0..L-1 of the directed operator on the symmetric oracle's
    geometry (Section 2.2's conditional semi-coarsening depends on the grid
    only; a fixed depth, levels >= 0).  galerkin: unit face factors (the
    P0^T H P0 coarse operators) instead of R10's."""
    p = params or O.MGParams()
    if p.levels < 0:
        raise ValueError("the nonsymmetric hierarchy takes a fixed depth (levels >= 0)")
    z = np.zeros_like(h)
    geo = O.build_hierarchy(z, z, z, np.ones_like(h), p)
    arr = [np.ascontiguousarray(a, dtype=np.float64) for a in (h, tx, ty, tz, txr, tyr, tzr)]
    return coarsen_all(NSLevel(*arr, geo[0]), geo, galerkin)


def coarsen_all(fine: NSLevel, geo, galerkin: bool = False):
    levels = [fine]
    for l in range(1, len(geo)):
        if galerkin:
            levels.append(coarsen(levels[-1], geo[l], 1.0, np.ones(geo[l].nlat)))
        else:
            levels.append(coarsen(levels[-1], geo[l]))
    return levels


def transposed(levels, galerkin: bool = False):
    """The hierarchy of H^T: the transpose of the finest operator, coarsened
    by the same rule (its couplings are the forward levels' swapped; its mass
    the sums of the fine column sums)."""
    return coarsen_all(transpose(levels[0]), [L.geo for L in levels], galerkin)


# --------------------------------------------------------------- V-cycle and solvers
def coarse_solve(lev: NSLevel, b, p: O.MGParams):
    """coarse_iters sweeps of Eq. (1) from zero on the coarsest level."""
    u = np.zeros_like(b)
    for _ in range(p.coarse_iters):
        u = smooth(lev, b, u, p.omega)
    return u


def vcycle(levels, b, params: O.MGParams | None = None, l: int = 0):
    """One V(nu1, nu2) cycle from zero (Section 2) on the given levels (pass
    transposed(levels) for the cycle of H^T)."""
    p = params or O.MGParams()
    lev = levels[l]
    if l == len(levels) - 1:
        return coarse_solve(lev, b, p)
    u = np.zeros_like(b)
    for _ in range(p.nu1):
        u = smooth(lev, b, u, p.omega)
    r = presmooth_residual(lev, b, u, p.omega) if p.nu1 == 1 else residual(lev, b, u)
    ec = vcycle(levels, O.restrict(lev.geo, r), p, l + 1)
    O.prolong_add(lev.geo, ec, u)
    for _ in range(p.nu2):
        u = smooth(lev, b, u, p.omega)
    return u


def _norm(x):
    return float(np.sqrt(np.dot(x.ravel(), x.ravel())))


def solve(levels, b, tol=1e-10, params: O.MGParams | None = None, maxit=None):
    """H x = b from x = 0 to ||b - H x|| <= tol ||b||: the stationary
    iteration x <- x + V(b - H x) (method "stationary") or BiCGStab right-
    preconditioned by the V-cycle (method "bicgstab": van der Vorst's
    iteration, shadow residual r^ = r_0, restarted from the true residual
    when the recursive one meets the tolerance without the true one).
    Returns (x, relative residual history, status)."""
    p = params or O.MGParams()
    maxit = p.maxit if maxit is None else maxit
    A = lambda v: apply(levels[0], v)
    M = lambda v: vcycle(levels, v, p)
    x = np.zeros_like(b)
    bn = _norm(b)
    hist = []
    if p.method == "stationary":
        for it in range(maxit + 1):
            r = b - A(x)
            rn = _norm(r)
            hist.append(rn / bn)
            if rn <= tol * bn:
                return x, hist, OK
            if it == maxit:
                break
            x = x + M(r)
        return x, hist, NOT_CONVERGED
    if p.method != "bicgstab":
        raise ValueError("nonsymmetric solves: method stationary or bicgstab")
    its = 0
    r0n = None
    while True:
        r = b - A(x)
        rn = _norm(r)
        r0n = rn if r0n is None else r0n
        hist.append(rn / bn)
        if rn <= tol * bn:
            return x, hist, OK
        if its >= maxit:
            return x, hist, NOT_CONVERGED
        rh = r.copy()
        rho_old = alpha = omega = 1.0
        v = np.zeros_like(b)
        pv = np.zeros_like(b)
        while its < maxit:
            its += 1
            rho = float(np.dot(rh.ravel(), r.ravel()))
            if rho == 0.0:
                break
            beta = (rho / rho_old) * (alpha / omega)
            pv = r + beta * (pv - omega * v)
            ph = M(pv)
            v = A(ph)
            rv = float(np.dot(rh.ravel(), v.ravel()))
            if rv == 0.0:
                break
            alpha = rho / rv
            s = r - alpha * v
            sh = M(s)
            t = A(sh)
            tt = float(np.dot(t.ravel(), t.ravel()))
            omega = float(np.dot(t.ravel(), s.ravel())) / tt if tt > 0 else 0.0
            x = x + alpha * ph + omega * sh
            r = s - omega * t
            rho_old = rho
            rn = _norm(r)
            if rn <= tol * bn or omega == 0.0:
                break
            hist.append(rn / bn)
            if rn > 1e6 * r0n:
                return x, hist, DIVERGED


def coeff_grad(lev: NSLevel, lam, x):
    """Gradient of L(x) with H x = b and lam = H^{-T} dL/dx, for the seven
    arrays: dL/dtheta = -lam^T (dH/dtheta) x.  h_c enters row c as h_c x_c;
    tx[c] row c as tx[c](x_c - x_E) and txr[c] row E as txr[c](x_E - x_c)
    (likewise y and z).  Pole, surface and top faces (fixed at zero) get
    zero.  Returns (gh, gtx, gty, gtz, gtxr, gtyr, gtzr)."""
    gh = -lam * x
    gtx = -lam * (x - east(x))
    gtxr = -east(lam) * (east(x) - x)
    gty = -lam * (x - north(x))
    gtyr = -north(lam) * (north(x) - x)
    gtz = -lam * (x - up(x))
    gtzr = -up(lam) * (up(x) - x)
    for g in (gty, gtyr):
        g[:, -1, :] = 0.0
    for g in (gtz, gtzr):
        g[-1] = 0.0
    return gh, gtx, gty, gtz, gtxr, gtyr, gtzr
