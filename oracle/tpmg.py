"""CPU oracle of the tensor-product multigrid solver (paper Sections 2.1-2.3).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the package's smoke check
and by the benchmark's CPU-baseline leg.  The CUDA library never imports it,
and it imports nothing from the library.  Inputs come from ``synthetic``.

Arithmetic lives in tpmg_oracle.c (double and float instances, built with
-ffp-contract=off); this module holds the hierarchy rule (Section 2.2), the
V-cycle recursion (Section 2 and Fig. 1), the multigrid solvers (Section 2:
the stationary iteration, and the V-cycle as preconditioner of conjugate
gradients), the mixed-precision refinement (Section 1's single-precision
remark), the gradient of the differentiable solve, in the order the method
states them, and the spectrum of H_z^{-1} H whose condition number Section
2.3's shallow-hierarchy argument rests on.

Pinned by tests/test_oracle_pins.py and tests/test_oracle_convergence.py; the
mixed-precision trajectory is pinned only by its convergence (parity unpinned
beyond that, no number in the paper).
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass, field

import numpy as np

from . import build as _build

_LIB = None

OK, NOT_CONVERGED = 0, 4


def _lib():
    global _LIB
    if _LIB is None:
        lib = ctypes.CDLL(_build.build())
        P = np.ctypeslib.ndpointer
        d = P(dtype=np.float64, flags="C_CONTIGUOUS")
        f = P(dtype=np.float32, flags="C_CONTIGUOUS")
        ip = P(dtype=np.int32, flags="C_CONTIGUOUS")
        I, S = ctypes.c_int, ctypes.c_size_t
        for sfx, a, real in (("_d", d, ctypes.c_double), ("_f", f, ctypes.c_float)):
            getattr(lib, "orc_apply" + sfx).argtypes = [I, I, I, a, a, a, a, a, a]
            getattr(lib, "orc_residual" + sfx).argtypes = [I, I, I, a, a, a, a, a, a, a]
            getattr(lib, "orc_presmooth_residual" + sfx).argtypes = [I, I, I, a, a, a, a, real, a]
            getattr(lib, "orc_smooth" + sfx).argtypes = [I, I, I, a, a, a, a, a, a, real, a]
            getattr(lib, "orc_column_solve_all" + sfx).argtypes = [I, I, I, a, a, a, a, a, a]
            getattr(lib, "orc_restrict" + sfx).argtypes = [I, I, I, I, ip, d, ip, d, a, a]
            getattr(lib, "orc_prolong_add" + sfx).argtypes = [I, I, I, I, ip, d, ip, d, a, a]
        lib.orc_dot.argtypes = [S, d, d]
        lib.orc_dot.restype = ctypes.c_double
        lib.orc_maxabs.argtypes = [S, d]
        lib.orc_maxabs.restype = ctypes.c_double
        lib.orc_coarsen_coeffs.argtypes = [I, I, I, I, ip, ip, ctypes.c_double, d,
                                           d, d, d, d, d, d, d, d]
        lib.orc_coeff_grad.argtypes = [I, I, I, d, d, d, d, d, d]
        lib.orc_num_threads.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def num_threads() -> int:
    return int(_lib().orc_num_threads())


@dataclass
class MGParams:
    """Readings of what the paper leaves open (listed in the design notes)."""
    levels: int = 0            # 0: coarsen down to the coarsest level (nlon >= 4);
    #                            Section 2.3's shallow hierarchy is levels=4; -1: stop at the
    #                            first level whose couplings are within iso_ratio (below)
    iso_ratio: float = 6.25    # levels=-1: largest (sum of horizontal couplings) / h allowed on
    #                            the coarsest level (4 faces at Section 2.3's nu^2 / 4^3 = 1.56)
    nu1: int = 1               # pre-smoothing sweeps, V(1,1)
    nu2: int = 1               # post-smoothing sweeps
    omega: float = 0.85        # Eq. (1) relaxation factor (value not printed; tuned)
    coarse_iters: int = 12     # Section 2.3's simple coarsest-grid iteration: block-Jacobi sweeps
    #                            (count not printed; measured), or PCG iterations
    coarse_method: str = "jacobi"  # coarsest-level solve: "jacobi" sweeps, "pcg" (CG
    #                                preconditioned by the column solves) or "chebyshev"
    #                                (Chebyshev steps on the column-solve preconditioner), from zero
    alpha_c: float = 0.6       # Section 2.2 anisotropy threshold (value not printed; tuned)
    method: str = "cg"         # outer iteration: "cg" (V-cycle-preconditioned CG), "stationary",
    #                            "bicgstab" (V-cycle-preconditioned) or "bicgstab_line" (BiCGStab
    #                            preconditioned by line_sweeps sweeps of Eq. (1): Section 1's solver)
    line_sweeps: int = 1       # bicgstab_line: sweeps of Eq. (1) per preconditioner application
    maxit: int = 200
    inner_tol: float = 5e-4    # mixed precision: FP32 inner relative tolerance per refinement step
    inner_maxit: int = 12      # mixed precision: FP32 inner iterations per refinement step


MIN_COARSE_NLON = 4


def auto_levels(nlon: int) -> int:
    """Number of levels when coarsening down to the coarsest level: halve the
    longitudes while the coarse grid keeps at least MIN_COARSE_NLON of them."""
    L = 1
    n = nlon
    while n % 2 == 0 and n // 2 >= MIN_COARSE_NLON:
        n //= 2
        L += 1
    return L


@dataclass
class Level:
    nlon: int
    nlat: int
    nz: int
    tx: np.ndarray
    ty: np.ndarray
    tz: np.ndarray
    h: np.ndarray
    south: np.ndarray          # row south edges (latitude, rad)
    north: np.ndarray          # row north edges
    # links to the next coarser level (None on the coarsest):
    row_of: np.ndarray | None = None   # fine row -> coarse row containing it
    nlat_c: int = 0
    top_row: np.ndarray | None = None  # coarse row -> its northern-most fine row
    j0: np.ndarray | None = None       # prolongation in latitude: fine row j takes
    w0: np.ndarray | None = None       #   w0[j] * coarse row j0[j]
    j1: np.ndarray | None = None       # + w1[j] * coarse row j1[j]  (j1 = -1: none)
    w1: np.ndarray | None = None
    scale: float = 1.0                 # FP32 copies hold scale * (FP64 coefficients)

    @property
    def shape(self):
        return (self.nz, self.nlat, self.nlon)

    @property
    def size(self):
        return self.nz * self.nlat * self.nlon

    @property
    def centres(self):
        return 0.5 * (self.south + self.north)

    def coeffs(self):
        return self.tx, self.ty, self.tz, self.h

    def links(self):
        return self.j0, self.w0, self.j1, self.w1


# --------------------------------------------------------------------- hierarchy
def fine_rows(nlat: int):
    """Level-0 row edges of the uniform lat-lon grid."""
    edges = -0.5 * np.pi + np.arange(nlat + 1) * (np.pi / nlat)
    edges[0], edges[-1] = -0.5 * np.pi, 0.5 * np.pi
    return edges[:-1].copy(), edges[1:].copy()


def coarsen_rows(south, north, nlon_coarse: int, alpha_c: float):
    """Conditional semi-coarsening of the latitude rows (Section 2.2).

    Longitude is always halved.  In each hemisphere the rows are visited from
    the equator towards the pole; rows q and q+1 are merged while the merged
    coarse cell keeps an anisotropy alpha = dx_lon / dx_lat =
    cos(theta_c) dlambda_coarse / (dtheta_q + dtheta_{q+1}) >= alpha_c
    (theta_c the centre of the merged row); from the first row where that
    fails, the remaining rows towards the pole stay single.  The southern
    hemisphere mirrors the northern one.

    Returns (row_of, coarse_south, coarse_north, top_row).
    """
    n = len(south)
    if n % 2:
        raise ValueError("row count must be even (mirror-symmetric hemispheres)")
    half = n // 2
    dlon_c = 2.0 * np.pi / nlon_coarse
    groups = []             # northern hemisphere: (first row, count)
    q, merging = half, True
    while q < n:
        if merging and q + 1 < n:
            th_s, th_n = south[q], north[q + 1]
            alpha = np.cos(0.5 * (th_s + th_n)) * dlon_c / (th_n - th_s)
            if alpha >= alpha_c:
                groups.append((q, 2))
                q += 2
                continue
            merging = False
        groups.append((q, 1))
        q += 1
    south_groups = [(n - 1 - (g + c - 1), c) for g, c in reversed(groups)]
    all_groups = south_groups + groups
    row_of = np.empty(n, dtype=np.int32)
    cs, cn, top = [], [], []
    for J, (g, c) in enumerate(all_groups):
        row_of[g:g + c] = J
        cs.append(south[g])
        cn.append(north[g + c - 1])
        top.append(g + c - 1)
    return row_of, np.array(cs), np.array(cn), np.array(top, dtype=np.int32)


def lat_interpolation(fine_centres, coarse_centres, row_of):
    """Linear interpolation in latitude between coarse row centres.

    A fine row whose centre coincides with its parent's (an unmerged row)
    takes the parent alone; otherwise it interpolates between the parent and
    the neighbouring coarse row on its side, by centre distance.  Beyond the
    outermost coarse centres (next to the poles) the parent is taken alone.
    """
    n, nc = len(fine_centres), len(coarse_centres)
    j0 = row_of.astype(np.int32).copy()
    w0 = np.ones(n)
    j1 = np.full(n, -1, dtype=np.int32)
    w1 = np.zeros(n)
    for j in range(n):
        J = int(row_of[j])
        d = fine_centres[j] - coarse_centres[J]
        if d == 0.0:
            continue
        Jn = J + 1 if d > 0 else J - 1
        if Jn < 0 or Jn >= nc:
            continue
        w = d / (coarse_centres[Jn] - coarse_centres[J])
        j1[j], w1[j], w0[j] = Jn, w, 1.0 - w
    return j0, w0, j1, w1


def horizontal_ratio(lev: Level) -> float:
    """The largest (sum of the four horizontal couplings) / h over a level:
    the square of the horizontal Courant number of Section 2.3 summed over
    the faces, 1 / mu - 1 for mu of hz_interval."""
    mu, _ = hz_interval(lev)
    return 1.0 / mu - 1.0


def build_hierarchy(tx, ty, tz, h, params: MGParams | None = None):
    """Levels 0..L-1 with rediscretised coarse coefficients (Sections 2.1-2.3).
    levels = -1: coarsen until a level's horizontal_ratio is at most
    iso_ratio (the coarse problem is then well conditioned, the premise of
    Section 2.3's shallow hierarchy), at most as deep as levels = 0."""
    p = params or MGParams()
    nz, nlat, nlon = h.shape
    L = p.levels if p.levels > 0 else auto_levels(nlon)
    if nlon % (1 << (L - 1)):
        raise ValueError("nlon must be divisible by 2^(levels-1)")
    s, n = fine_rows(nlat)
    levels = [Level(nlon, nlat, nz, *(np.ascontiguousarray(a, dtype=np.float64)
                                      for a in (tx, ty, tz, h)), s, n)]
    lib = _lib()
    for _ in range(1, L):
        f = levels[-1]
        nlon_c = f.nlon // 2
        row_of, cs, cn, top = coarsen_rows(f.south, f.north, nlon_c, p.alpha_c)
        nlat_c = len(cs)
        cc = 0.5 * (cs + cn)
        f.row_of, f.nlat_c, f.top_row = row_of, nlat_c, top
        f.j0, f.w0, f.j1, f.w1 = lat_interpolation(f.centres, cc, row_of)
        fc = f.centres
        sy = np.zeros(nlat_c)
        for J in range(nlat_c - 1):
            t = top[J]
            sy[J] = (fc[t + 1] - fc[t]) / (cc[J + 1] - cc[J])
        shape_c = (nz, nlat_c, nlon_c)
        txc, tyc, tzc, hc = (np.empty(shape_c) for _ in range(4))
        lib.orc_coarsen_coeffs(f.nlon, f.nlat, nz, nlat_c, row_of, top, 0.5, sy,
                               f.tx, f.ty, f.tz, f.h, txc, tyc, tzc, hc)
        levels.append(Level(nlon_c, nlat_c, nz, txc, tyc, tzc, hc, cs, cn))
        if p.levels < 0 and horizontal_ratio(levels[-1]) <= p.iso_ratio:
            break
    return levels


def float_levels(levels):
    """FP32 copies of every level, rounded from FP64 after scaling all
    coefficients by one power of two (exact) so that the largest becomes
    O(1): FP32's range then holds every product of the column solves."""
    big = max(float(np.max(a)) for lev in levels for a in lev.coeffs())
    _, ex = np.frexp(big)
    scale = float(np.ldexp(1.0, -int(ex)))
    out = []
    for lev in levels:
        c = [np.ascontiguousarray(a * scale, dtype=np.float32) for a in lev.coeffs()]
        out.append(Level(lev.nlon, lev.nlat, lev.nz, *c, lev.south, lev.north,
                         lev.row_of, lev.nlat_c, lev.top_row,
                         lev.j0, lev.w0, lev.j1, lev.w1, scale))
    return out


# ------------------------------------------------------------------- primitives
def _sfx(a):
    return "_d" if a.dtype == np.float64 else "_f"


def apply(lev: Level, u):
    y = np.empty_like(u)
    getattr(_lib(), "orc_apply" + _sfx(u))(lev.nlon, lev.nlat, lev.nz, *lev.coeffs(), u, y)
    return y


def residual(lev: Level, b, u):
    r = np.empty_like(u)
    getattr(_lib(), "orc_residual" + _sfx(u))(lev.nlon, lev.nlat, lev.nz, *lev.coeffs(), b, u, r)
    return r


def presmooth_residual(lev: Level, b, u, omega):
    """The residual b - H u of u = omega H_z^{-1} b, the sweep of Eq. (1) from
    a zero guess, written without the column couplings it cancels: since
    H_z u = omega b, b - H u = (1 - omega) b - dH u = (1 - omega) b + the sum
    over the four horizontal faces of T_f u_nb(f).  Evaluated in u's
    precision, the terms added in the order east, west, north, south."""
    r = np.empty_like(u)
    om1 = u.dtype.type(1.0) - u.dtype.type(omega)
    getattr(_lib(), "orc_presmooth_residual" + _sfx(u))(lev.nlon, lev.nlat, lev.nz, lev.tx,
                                                         lev.ty, b, u, om1, r)
    return r


def column_solve(lev: Level, r):
    x = np.empty_like(r)
    getattr(_lib(), "orc_column_solve_all" + _sfx(r))(lev.nlon, lev.nlat, lev.nz,
                                                        *lev.coeffs(), r, x)
    return x


def smooth(lev: Level, b, u, omega: float, work=None):
    """One sweep of Eq. (1), in place on u."""
    if work is None:
        work = np.empty_like(u)
    getattr(_lib(), "orc_smooth" + _sfx(u))(lev.nlon, lev.nlat, lev.nz, *lev.coeffs(),
                                             b, u, omega, work)


def restrict(lev: Level, r):
    bc = np.empty((lev.nz, lev.nlat_c, lev.nlon // 2), dtype=r.dtype)
    getattr(_lib(), "orc_restrict" + _sfx(r))(lev.nlon, lev.nlat, lev.nz, lev.nlat_c,
                                               *lev.links(), r, bc)
    return bc


def prolong_add(lev: Level, ec, u):
    getattr(_lib(), "orc_prolong_add" + _sfx(u))(lev.nlon, lev.nlat, lev.nz, lev.nlat_c,
                                                  *lev.links(), ec, u)


def dot(x, y) -> float:
    """Inner product accumulated in FP64, serial index order."""
    x = np.ascontiguousarray(x, dtype=np.float64).ravel()
    y = np.ascontiguousarray(y, dtype=np.float64).ravel()
    return float(_lib().orc_dot(x.size, x, y))


def norm2(x) -> float:
    return float(np.sqrt(dot(x, x)))


# --------------------------------------------------------------------- coarsest level
def coarse_pcg(lev: Level, b, iters: int):
    """Conjugate gradients on one level from a zero guess, preconditioned by
    the column solves of Eq. (1) (z = H_z^{-1} r: a sweep from zero with
    omega = 1), exactly `iters` iterations: the conjugate-gradient form of
    the coarsest-grid iteration of Section 2.3.  Scalars in FP64, vectors in
    b's precision (x += alpha d, r -= alpha H d, d = z + beta d in that
    precision).  A zero <r, z> or <d, H d> ends it (exact solution reached)."""
    one = b.dtype.type(1.0)
    x = np.zeros_like(b)
    r = b.copy()
    z = np.zeros_like(b)
    smooth(lev, r, z, one)
    d = z.copy()
    rz = dot(r, z)
    for it in range(iters):
        q = apply(lev, d)
        dq = dot(d, q)
        if rz == 0.0 or dq == 0.0:
            break
        alpha = b.dtype.type(rz / dq)
        x += alpha * d
        r -= alpha * q
        if it + 1 == iters:
            break
        z = np.zeros_like(b)
        smooth(lev, r, z, one)
        rz_new = dot(r, z)
        beta = b.dtype.type(rz_new / rz)
        rz = rz_new
        d = z + beta * d
    return x


def hz_interval(lev: Level):
    """An interval [mu, 2] holding the spectrum of H_z^{-1} H.  2 H_z - H =
    H_z - dH is diagonally dominant with a positive diagonal, so lambda < 2;
    u' H u = sum h u^2 + (vertical and horizontal couplings, both >= 0) and
    u' H_z u = sum (h + horizontal couplings) u^2 + (the same vertical
    part), so lambda >= mu = min over cells of h / (h + the four horizontal
    couplings).  Computed in FP64 from the level's coefficients (a FP32
    level holds them scaled, which leaves the ratios unchanged)."""
    h = lev.h.astype(np.float64)
    tx = lev.tx.astype(np.float64)
    ty = lev.ty.astype(np.float64)
    hor = tx + np.roll(tx, 1, axis=2) + ty
    hor[:, 1:, :] += ty[:, :-1, :]
    return float(np.min(h / (h + hor))), 2.0


def coarse_chebyshev(lev: Level, b, iters: int):
    """Chebyshev iteration from a zero guess preconditioned by the column
    solves (M = H_z), exactly `iters` steps, on the interval [mu, 2] of
    hz_interval: a fixed polynomial in H_z^{-1} H, so the coarsest-level
    solve (Section 2.3's simple iteration, here polynomially accelerated)
    stays a fixed symmetric linear operator.  With theta = (2 + mu) / 2,
    delta = (2 - mu) / 2, sigma = theta / delta (scalars in FP64):
        r_0 = b, d_0 = M^{-1} r_0 / theta, rho_0 = 1 / sigma
        x_{k+1} = x_k + d_k;  r_{k+1} = r_k - H d_k
        rho_{k+1} = 1 / (2 sigma - rho_k)
        d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1} / delta) M^{-1} r_{k+1}
    The error after m steps is T_m((theta - H_z^{-1} H) / delta) / T_m(sigma)
    times the initial error (T_m the Chebyshev polynomial).  Vectors in b's
    precision; the column solves are sweeps from zero with omega = 1."""
    mu, lam = hz_interval(lev)
    theta, delta = 0.5 * (lam + mu), 0.5 * (lam - mu)
    sigma = theta / delta
    dt = b.dtype.type
    one = dt(1.0)
    x = np.zeros_like(b)
    r = b.copy()
    z = np.zeros_like(b)
    smooth(lev, r, z, one)
    d = (z * dt(1.0 / theta)).astype(b.dtype)
    rho = 1.0 / sigma
    for it in range(iters):
        x += d
        if it + 1 == iters:
            break
        r = residual(lev, r, d)             # r - H d
        z = np.zeros_like(b)
        smooth(lev, r, z, one)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = (dt(rho_new * rho) * d + dt(2.0 * rho_new / delta) * z).astype(b.dtype)
        rho = rho_new
    return x


def coarse_solve(lev: Level, b, p: MGParams):
    """The coarsest-level solve of the V-cycle from a zero guess (Section
    2.3): coarse_iters block-Jacobi sweeps, PCG iterations or Chebyshev
    steps."""
    if p.coarse_method == "pcg":
        return coarse_pcg(lev, b, p.coarse_iters)
    if p.coarse_method == "chebyshev":
        return coarse_chebyshev(lev, b, p.coarse_iters)
    om = np.float32(p.omega) if b.dtype == np.float32 else p.omega
    u = np.zeros_like(b)
    work = np.empty_like(b)
    for _ in range(p.coarse_iters):
        smooth(lev, b, u, om, work)
    return u


# --------------------------------------------------------------------- V-cycle
def vcycle(levels, b, params: MGParams | None = None, l: int = 0):
    """One V(nu1, nu2) cycle from a zero initial guess (Section 2, Fig. 1):
    smooth, restrict the residual, recurse, prolongate the correction, smooth.
    On the coarsest level: coarse_solve (Section 2.3's simple iteration on
    the coarsest grid)."""
    p = params or MGParams()
    lev = levels[l]
    if l == len(levels) - 1:
        return coarse_solve(lev, b, p)
    om = np.float32(p.omega) if b.dtype == np.float32 else p.omega
    u = np.zeros_like(b)
    work = np.empty_like(b)
    for _ in range(p.nu1):
        smooth(lev, b, u, om, work)
    # after a single sweep from zero the residual needs no column couplings
    r = presmooth_residual(lev, b, u, om) if p.nu1 == 1 else residual(lev, b, u)
    ec = vcycle(levels, restrict(lev, r), p, l + 1)
    prolong_add(lev, ec, u)
    for _ in range(p.nu2):
        smooth(lev, b, u, om, work)
    return u


def solve_stationary(levels, b, tol, params, x0=None, maxit=None):
    """x <- x + V(b - H x) until ||b - H x||_2 <= tol ||b||_2 (Section 2)."""
    p = params
    maxit = p.maxit if maxit is None else maxit
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=b.dtype, copy=True)
    bn = norm2(b)
    hist = []
    for it in range(maxit + 1):
        r = residual(levels[0], b, x)
        rn = norm2(r)
        hist.append(rn / bn if bn > 0 else 0.0)
        if rn <= tol * bn:
            return x, hist, OK
        if it == maxit:
            break
        x += vcycle(levels, r, p)
    return x, hist, NOT_CONVERGED


def solve_cg(levels, b, tol, params, x0=None, maxit=None):
    """Conjugate gradients preconditioned by one V-cycle (H and the V-cycle
    are symmetric positive definite).  Scalars in FP64; vectors in b's
    precision.  Stops on the recursively updated residual, then confirms
    with the true residual (restarting from x if the two disagree)."""
    p = params
    maxit = p.maxit if maxit is None else maxit
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=b.dtype, copy=True)
    bn = norm2(b)
    hist = []
    its = 0
    while True:
        r = residual(levels[0], b, x)
        rn = norm2(r)
        hist.append(rn / bn if bn > 0 else 0.0)
        if rn <= tol * bn:
            return x, hist, OK
        if its >= maxit:
            return x, hist, NOT_CONVERGED
        z = vcycle(levels, r, p)
        d = z.copy()
        rz = dot(r, z)
        while its < maxit:
            its += 1
            Ad = apply(levels[0], d)
            alpha = rz / dot(d, Ad)
            x += alpha * d
            r -= alpha * Ad
            rn = norm2(r)
            if rn <= tol * bn:
                break
            hist.append(rn / bn)
            z = vcycle(levels, r, p)
            rz_new = dot(r, z)
            beta = rz_new / rz
            rz = rz_new
            d = z + beta * d


def line_relaxation(lev: Level, r, sweeps: int, omega: float):
    """The preconditioner of the BiCGStab solver the paper's multigrid
    replaced (Section 1: BiCGStab preconditioned with vertical line
    relaxation; Section 2.1: the iteration of Eq. (1) preconditions
    BiCGStab in the original model): `sweeps` sweeps of Eq. (1) from a zero
    guess on r."""
    om = r.dtype.type(omega)
    u = np.zeros_like(r)
    work = np.empty_like(r)
    for _ in range(sweeps):
        smooth(lev, r, u, om, work)
    return u


def solve_bicgstab(levels, b, tol, params, x0=None, maxit=None, precond: str = "line",
                   sweeps: int = 1):
    """BiCGStab (van der Vorst's stabilised bi-conjugate gradients) with right
    preconditioning M: precond "line" is the vertical line relaxation of
    Eq. (1) (`sweeps` sweeps from zero, the solver of Section 1 that the
    multigrid replaced), "mg" one V-cycle.  Per iteration, with the shadow
    residual rh = r_0:
        rho = <rh, r>;  beta = (rho / rho_old) (alpha / w)
        p = r + beta (p - w v);  ph = M p;  v = H ph;  alpha = rho / <rh, v>
        s = r - alpha v  (stop if ||s|| <= tol ||b||: x += alpha ph)
        sh = M s;  t = H sh;  w = <t, s> / <t, t>
        x += alpha ph + w sh;  r = s - w t
    Scalars in FP64, vectors in b's precision; stops on the recursively
    updated residual, then confirms with the true residual (restarting from
    x, with a new shadow residual, if they disagree or on a breakdown
    rho = 0, <rh, v> = 0 or <t, t> = 0).  One iteration = two
    preconditioner applications and two operator applications.  Returns
    (x, rel_history, status)."""
    p = params
    maxit = p.maxit if maxit is None else maxit
    dt = b.dtype.type
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=b.dtype, copy=True)
    bn = norm2(b)
    hist = []
    its = 0

    def M(v):
        if precond == "mg":
            return vcycle(levels, v, p)
        return line_relaxation(levels[0], v, sweeps, p.omega)

    while True:
        r = residual(levels[0], b, x)
        rn = norm2(r)
        hist.append(rn / bn if bn > 0 else 0.0)
        if rn <= tol * bn:
            return x, hist, OK
        if its >= maxit:
            return x, hist, NOT_CONVERGED
        rh = r.copy()
        rho_old = alpha = w = 1.0
        v = np.zeros_like(b)
        pv = np.zeros_like(b)
        while its < maxit:
            its += 1
            rho = dot(rh, r)
            if rho == 0.0:
                break                                   # breakdown: restart
            beta = (rho / rho_old) * (alpha / w)
            pv = r + dt(beta) * (pv - dt(w) * v)
            ph = M(pv)
            v = apply(levels[0], ph)
            rv = dot(rh, v)
            if rv == 0.0:
                break
            alpha = rho / rv
            s = r - dt(alpha) * v
            if norm2(s) <= tol * bn:
                x += dt(alpha) * ph
                break                                   # confirm with the true residual
            sh = M(s)
            t = apply(levels[0], sh)
            tt = dot(t, t)
            if tt == 0.0:
                x += dt(alpha) * ph
                break
            w = dot(t, s) / tt
            x += dt(alpha) * ph + dt(w) * sh
            r = s - dt(w) * t
            rho_old = rho
            rn = norm2(r)
            if rn <= tol * bn or w == 0.0:
                break                                   # confirm with the true residual
            hist.append(rn / bn)


def solve(levels, b, tol: float = 1e-10, x0=None, params: MGParams | None = None,
          maxit: int | None = None):
    """Multigrid solve of H x = b to ||b - H x||_2 <= tol ||b||_2.
    Returns (x, rel_history, status)."""
    p = params or MGParams()
    if p.method == "stationary":
        return solve_stationary(levels, b, tol, p, x0, maxit)
    if p.method == "bicgstab":
        return solve_bicgstab(levels, b, tol, p, x0, maxit, precond="mg")
    if p.method == "bicgstab_line":
        return solve_bicgstab(levels, b, tol, p, x0, maxit, precond="line",
                              sweeps=p.line_sweeps)
    return solve_cg(levels, b, tol, p, x0, maxit)


def solve_mixed(levels, b, tol: float = 1e-10, params: MGParams | None = None,
                levels32=None, maxit: int | None = None, track=None):
    """FP32 multigrid inside FP64 iterative refinement.

    Outer loop in FP64: r = b - H x, stop when ||r||_2 <= tol ||b||_2; scale r
    by a power of two s (exact; keeps FP32 clear of under/overflow) and round
    to FP32; inner: solve (c H) e = r / s in FP32 storage and arithmetic
    (FP64 scalars) to max(inner_tol, 0.3 tol / (||r|| / ||b||)) (at most 0.5),
    at most inner_maxit iterations, with the same outer iteration as the FP64
    solver; update x <- x + c s e in FP64,
    c the power-of-two scale of the FP32 coefficient copies.
    ``track(x)`` is called after every update.  Returns (x, rel_history, status)."""
    p = params or MGParams()
    maxit = p.maxit if maxit is None else maxit
    l32 = levels32 if levels32 is not None else float_levels(levels)
    x = np.zeros_like(b)
    bn = norm2(b)
    hist = []
    for it in range(maxit + 1):
        r = residual(levels[0], b, x)
        rn = norm2(r)
        hist.append(rn / bn if bn > 0 else 0.0)
        if rn <= tol * bn:
            return x, hist, OK
        if it == maxit:
            break
        refine_correct(l32, x, r, rn, bn, tol, p)
        if track is not None:
            track(x)
    return x, hist, NOT_CONVERGED


def refine_correct(levels32, x, r, rn, bn, tol, p: MGParams):
    """The correction of one refinement step of solve_mixed, in place on the
    FP64 iterate x given its FP64 residual r (norm rn; bn = ||b||): scale r by
    the power of two s at its largest magnitude, round to FP32, solve
    (c H) e = r / s with the FP32 multigrid to the inner tolerance, and add
    c s e in FP64."""
    c = levels32[0].scale
    _, ex = np.frexp(np.max(np.abs(r)))
    s = float(np.ldexp(1.0, int(ex)))
    r32 = (r / s).astype(np.float32)
    # no further than the outer target still needs (safety 0.3), at most 0.5
    itol = min(max(p.inner_tol, 0.3 * tol / (rn / bn)), 0.5)
    e, _, _ = solve(levels32, r32, itol, params=p, maxit=p.inner_maxit)
    x += (c * s) * e.astype(np.float64)


# ------------------------------------------------------------------- gradient
def coeff_grad(lev: Level, lam, x):
    """(dL/dh, dL/dtx, dL/dty, dL/dtz) given the adjoint lambda and solution x."""
    out = [np.empty_like(x) for _ in range(4)]
    _lib().orc_coeff_grad(lev.nlon, lev.nlat, lev.nz, lam, x, *out)
    return tuple(out)


def solve_with_grad(levels, b, dLdx_fn, tol=1e-13, params=None):
    """x = H^{-1} b, lambda = H^{-T} dL/dx (H is symmetric: same hierarchy),
    returns x, dL/db = lambda and the coefficient gradients."""
    x, _, _ = solve(levels, b, tol, params=params)
    g = dLdx_fn(x)
    lam, _, _ = solve(levels, g, tol, params=params)
    gh, gtx, gty, gtz = coeff_grad(levels[0], lam, x)
    return x, dict(b=lam, h=gh, tx=gtx, ty=gty, tz=gtz)


# ----------------------------------------------- condition number (Section 2.3)
def sparse_operator(lev: Level):
    """H of one level as a scipy CSR matrix, read off the oracle's own apply:
    every cell's stencil reaches layers k-1..k+1, rows j-1..j+1 and
    longitudes i-1..i+1 (mod nlon), so the 36 colourings (k mod 3, j mod 3,
    i mod 4) give each stencil at most one probed cell per colour (nlon a
    multiple of 4), and H applied to a colour's indicator holds column
    entries H[row, col] for the probed cells col.  Tiny or moderate grids."""
    import scipy.sparse as sp
    nz, nlat, nlon = lev.shape
    if nlon % 4:
        raise ValueError("probing needs nlon divisible by 4")
    K, J, I = np.meshgrid(np.arange(nz), np.arange(nlat), np.arange(nlon), indexing="ij")
    colour = (K % 3) * 12 + (J % 3) * 4 + (I % 4)
    idx = np.arange(lev.size).reshape(lev.shape)
    rows, cols, vals = [], [], []
    for c in range(36):
        y = apply(lev, (colour == c).astype(np.float64))
        for dk, dj, di in ((0, 0, 0), (1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0),
                           (0, 0, 1), (0, 0, -1)):
            kk, jj, ii = K + dk, J + dj, (I + di) % nlon
            ok = (kk >= 0) & (kk < nz) & (jj >= 0) & (jj < nlat)
            kk, jj = np.clip(kk, 0, nz - 1), np.clip(jj, 0, nlat - 1)
            m = ok & (colour[kk, jj, ii] == c)
            rows.append(idx[m])
            cols.append(idx[kk, jj, ii][m])
            vals.append(y[m])
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(lev.size, lev.size)).tocsr()
    A.eliminate_zeros()
    return A


def column_part(A, lev: Level):
    """H_z of Section 2.1: the entries of H that couple cells of one vertical
    column (its diagonal and the couplings between layers)."""
    import scipy.sparse as sp
    C = A.tocoo()
    ncol = lev.nlat * lev.nlon
    m = (C.row % ncol) == (C.col % ncol)
    return sp.csr_matrix((C.data[m], (C.row[m], C.col[m])), shape=A.shape)


def row_band(lev: Level, j0: int, j1: int) -> Level:
    """Rows j0..j1-1 of a level as a level of their own, with zero-flux faces
    at the band's southern and northern edges (the couplings to the rows
    outside are dropped, so the constant stays the smoothest mode)."""
    s = slice(j0, j1)
    ty = lev.ty[:, s, :].copy()
    ty[:, -1, :] = 0.0
    cut = lambda a: np.ascontiguousarray(a[:, s, :])
    return Level(lev.nlon, j1 - j0, lev.nz, cut(lev.tx), ty, cut(lev.tz), cut(lev.h),
                 lev.south[s].copy(), lev.north[s].copy())


def hz_spectrum(lev: Level, tol: float = 1e-9):
    """Extreme eigenvalues (lambda_min, lambda_max) of H_z^{-1} H, whose ratio
    is the condition number that Section 2.3 says governs the block-Jacobi
    iteration of Eq. (1): the generalised symmetric problem H v = lambda H_z v
    by Lanczos (scipy's eigsh, relative accuracy tol), the smallest by
    shift-invert about 0."""
    import scipy.sparse.linalg as spla
    A = sparse_operator(lev)
    Z = column_part(A, lev)
    lmax = spla.eigsh(A, k=1, M=Z, which="LA", tol=tol, return_eigenvectors=False)[0]
    lmin = spla.eigsh(A, k=1, M=Z, sigma=0.0, which="LM", tol=tol,
                      return_eigenvectors=False)[0]
    return float(lmin), float(lmax)


def courant_squared(lmin: float, horizontal_faces: int = 4) -> float:
    """The squared horizontal Courant number read off lambda_min of
    H_z^{-1} H.  For the constant mode of a band with zero-flux edges H u =
    h u and H_z u = (h + sum of the horizontal couplings) u, so
    1 / lambda_min - 1 = (sum of the four horizontal couplings) / h, which is
    4 nu^2 on a grid of square cells (t_x / h = t_y / h = nu^2 at the
    equator of the generator): nu^2 = (1 / lambda_min - 1) / 4."""
    return (1.0 / lmin - 1.0) / horizontal_faces


def dense_operator(lev: Level) -> np.ndarray:
    """H as a dense matrix, column c = H e_c (tiny grids only)."""
    n = lev.size
    A = np.empty((n, n))
    e = np.zeros(lev.shape)
    for c in range(n):
        e.flat[c] = 1.0
        A[:, c] = apply(lev, e).ravel()
        e.flat[c] = 0.0
    return A
