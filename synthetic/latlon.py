"""Cell-centred finite-volume lat-lon shell grid and the seeded coefficient fields.

The pressure-correction system of the paper (Section 2) is H u = b with H a
sparse operator of Laplacian type on a latitude-longitude grid with a strongly
stretched vertical (Section 1: high aspect ratio; Section 2.2: the
anisotropy alpha(theta) = dx_lon / dx_lat of the lat-lon grid).  The paper
prints no discretisation, so this module fixes one (a reading, documented in
the design notes):

* longitudes  lambda_i = (i + 1/2) dlambda,   dlambda = 2 pi / nlon  (periodic)
* latitudes   theta_j  = -pi/2 + (j + 1/2) dtheta,  dtheta = pi / nlat
* radial faces r_k = R + top (k / nz)^2, k = 0..nz  (quadratic stretching)

Each cell carries a Helmholtz term h = V (its exact shell-sector volume) and
each face a coupling T = K * area / distance, K = (nu R dlambda)^2 with the
horizontal Courant number nu = 10 (Section 2.3), so that T_lon / h is close
to nu^2 / cos^2(theta).  Faces on the poles, the surface and the model top
have zero area, hence T = 0 there (no-flux boundaries).

Coefficients are then multiplied by exp(sigma * g_c) with g a seeded N(0,1)
field smoothed by a 3-point box filter along lon (periodic), then lat, then
height (edges average the available neighbours).  A face gets the geometric
mean exp(sigma * (g_c1 + g_c2) / 2) of its two cells, which keeps H
symmetric.  The right-hand side is i.i.d. uniform[-1, 1], drawn after g from
the same generator.

Array layout (shared by oracle and library): float64, C order, shape
[nz][nlat][nlon]; index (k, j, i).
  tx[k,j,i] : face between lon cells i and i+1 (mod nlon)
  ty[k,j,i] : face between lat rows j and j+1; ty[:, nlat-1, :] = 0 (north pole)
  tz[k,j,i] : face between layers k and k+1; tz[nz-1] = 0 (model top)
  h [k,j,i] : Helmholtz diagonal term
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

EARTH_RADIUS_M = 6371.0e3
MODEL_TOP_M = 80.0e3
COURANT_NU = 10.0


@dataclass(frozen=True)
class ShellGrid:
    nlon: int
    nlat: int
    nz: int
    radius: float = EARTH_RADIUS_M
    top: float = MODEL_TOP_M

    @property
    def dlon(self) -> float:
        return 2.0 * np.pi / self.nlon

    @property
    def dlat(self) -> float:
        return np.pi / self.nlat

    def lat_faces(self) -> np.ndarray:
        """theta_{j-1/2}, j = 0..nlat (the poles are exactly -pi/2 and pi/2)."""
        t = -0.5 * np.pi + np.arange(self.nlat + 1) * self.dlat
        t[0], t[-1] = -0.5 * np.pi, 0.5 * np.pi
        return t

    def lat_centres(self) -> np.ndarray:
        return -0.5 * np.pi + (np.arange(self.nlat) + 0.5) * self.dlat

    def lon_centres(self) -> np.ndarray:
        return (np.arange(self.nlon) + 0.5) * self.dlon

    def r_faces(self) -> np.ndarray:
        k = np.arange(self.nz + 1, dtype=np.float64)
        return self.radius + self.top * (k / self.nz) ** 2

    def r_centres(self) -> np.ndarray:
        rf = self.r_faces()
        return 0.5 * (rf[:-1] + rf[1:])

    def _sin_lat_faces(self) -> np.ndarray:
        s = np.sin(self.lat_faces())
        s[0], s[-1] = -1.0, 1.0
        return s

    def _cos_lat_faces(self) -> np.ndarray:
        c = np.cos(self.lat_faces())
        c[0], c[-1] = 0.0, 0.0
        return c

    def volumes(self) -> np.ndarray:
        """[nz, nlat] exact shell-sector volumes (independent of longitude)."""
        rf = self.r_faces()
        ds = np.diff(self._sin_lat_faces())
        dr3 = (rf[1:] ** 3 - rf[:-1] ** 3) / 3.0
        return dr3[:, None] * (self.dlon * ds)[None, :]

    def geometry_coefficients(self, K: float):
        """Unperturbed (tx, ty, tz, h) on [nz, nlat] (no lon dependence).

        tx: east faces, area dtheta (r_{k+1}^2 - r_k^2)/2, distance r_c cos(theta_j) dlambda
        ty: north faces, area cos(theta_{j+1/2}) dlambda (r_{k+1}^2 - r_k^2)/2,
            distance r_c dtheta; zero on the north pole face
        tz: upper faces, area r_{k+1}^2 dlambda (sin theta_{j+1/2} - sin theta_{j-1/2}),
            distance between layer centres; zero on the model top
        """
        rf, rc = self.r_faces(), self.r_centres()
        half_dr2 = 0.5 * (rf[1:] ** 2 - rf[:-1] ** 2)              # [nz]
        cos_c = np.cos(self.lat_centres())                          # [nlat]
        cos_f = self._cos_lat_faces()                               # [nlat+1]
        ds = np.diff(self._sin_lat_faces())                         # [nlat]

        ax = self.dlat * half_dr2[:, None] * np.ones(self.nlat)[None, :]
        dx = rc[:, None] * cos_c[None, :] * self.dlon
        tx = K * ax / dx

        ay = cos_f[None, 1:] * self.dlon * half_dr2[:, None]        # north face of row j
        dy = rc[:, None] * self.dlat * np.ones(self.nlat)[None, :]
        ty = K * ay / dy
        ty[:, -1] = 0.0

        tz = np.zeros((self.nz, self.nlat))
        if self.nz > 1:
            az = rf[1:-1, None] ** 2 * self.dlon * ds[None, :]      # faces k+1, k = 0..nz-2
            dz = np.diff(rc)[:, None]
            tz[:-1] = K * az / dz
        h = self.volumes()
        return tx, ty, tz, h


def box_filter_3pt(g: np.ndarray, axis: int, periodic: bool) -> np.ndarray:
    """3-point running mean along one axis; non-periodic edges average the
    neighbours that exist."""
    n = g.shape[axis]
    if n == 1:
        return g.copy()
    if periodic:
        return (np.roll(g, 1, axis=axis) + g + np.roll(g, -1, axis=axis)) / 3.0
    out = np.empty_like(g)
    sl = [slice(None)] * g.ndim

    def s(a, b):
        sl2 = list(sl)
        sl2[axis] = slice(a, b)
        return tuple(sl2)

    out[s(1, n - 1)] = (g[s(0, n - 2)] + g[s(1, n - 1)] + g[s(2, n)]) / 3.0
    out[s(0, 1)] = (g[s(0, 1)] + g[s(1, 2)]) / 2.0
    out[s(n - 1, n)] = (g[s(n - 2, n - 1)] + g[s(n - 1, n)]) / 2.0
    return out


def make_problem(nlon: int, nlat: int, nz: int, sigma: float, seed: int,
                 nu: float = COURANT_NU, radius: float = EARTH_RADIUS_M,
                 top: float = MODEL_TOP_M, K: float | None = None,
                 with_rhs: bool = True) -> dict:
    """Seeded coefficient fields and right-hand side, all float64 [nz, nlat, nlon].

    Returns dict(tx, ty, tz, h, b, grid, K).  ``K`` defaults to
    (nu * R * dlambda)^2; pass it explicitly to keep the continuous operator
    fixed across resolutions.
    """
    grid = ShellGrid(nlon, nlat, nz, radius, top)
    if K is None:
        K = (nu * radius * grid.dlon) ** 2
    tx2, ty2, tz2, h2 = grid.geometry_coefficients(K)
    shape = (nz, nlat, nlon)
    rng = np.random.default_rng(seed)

    def bcast(a):
        return np.ascontiguousarray(np.broadcast_to(a[:, :, None], shape))

    if sigma != 0.0:
        g = rng.standard_normal(shape)
        g = box_filter_3pt(g, axis=2, periodic=True)
        g = box_filter_3pt(g, axis=1, periodic=False)
        g = box_filter_3pt(g, axis=0, periodic=False)
        g *= sigma                                       # sigma * g_c
        h = np.exp(g)
        h *= h2[:, :, None]
        tx = np.exp(0.5 * (g + np.roll(g, -1, axis=2)))
        tx *= tx2[:, :, None]
        ty = np.zeros(shape)
        if nlat > 1:
            ty[:, :-1, :] = np.exp(0.5 * (g[:, :-1, :] + g[:, 1:, :]))
            ty[:, :-1, :] *= ty2[:, :-1, None]
        tz = np.zeros(shape)
        if nz > 1:
            tz[:-1] = np.exp(0.5 * (g[:-1] + g[1:]))
            tz[:-1] *= tz2[:-1, :, None]
        del g
    else:
        rng.standard_normal(shape)  # keep the draw order identical
        h, tx, ty, tz = bcast(h2), bcast(tx2), bcast(ty2), bcast(tz2)
    out = dict(tx=tx, ty=ty, tz=tz, h=h, grid=grid, K=K)
    if with_rhs:
        out["b"] = rng.uniform(-1.0, 1.0, shape)
    return out


# Workloads, named by what they are.  Seeds: base + member.
WORKLOADS = {
    # plain FP64 solve whose oracle run finishes in seconds
    "latlon_64x32x16": dict(nlon=64, nlat=32, nz=16, sigma=0.1, seed_base=1000),
    # mixed precision vs FP64, ~55M unknowns
    "latlon_1024x768x70": dict(nlon=1024, nlat=768, nz=70, sigma=0.1, seed_base=2000),
    # operational size, ~124M unknowns, multiplier std 0.2
    "latlon_1536x1152x70": dict(nlon=1536, nlat=1152, nz=70, sigma=0.2, seed_base=3000),
    # differentiable solve
    "latlon_256x128x32": dict(nlon=256, nlat=128, nz=32, sigma=0.1, seed_base=4000),
}

# Ensemble of 24 uneven systems: (count, nlon, nlat, nz)
ENSEMBLE_MEMBERS = [(8, 256, 192, 70), (8, 512, 384, 70), (6, 1024, 768, 70), (2, 1536, 1152, 70)]
ENSEMBLE_SEED_BASE = 5000


def workload_seed(name: str, member: int = 0) -> int:
    if name == "ensemble":
        return ENSEMBLE_SEED_BASE + member
    return WORKLOADS[name]["seed_base"] + member


def make_ns_problem(nlon: int, nlat: int, nz: int, sigma: float, seed: int, pe: float = 0.3,
                    **kw) -> dict:
    """A nonsymmetric system: make_problem's operator plus upwind transport by
    a seeded divergence-free flow (a model of the advective terms that make
    the operational Helmholtz problem nonsymmetric).

    Face volume fluxes come from two stream functions on cell corners, one in
    the lon-lat plane (psi1 [nz, nlat+1, nlon], zero on the pole corners) and
    one in the lon-height plane (psi2 [nz+1, nlat, nlon], zero at the surface
    and the top):
      Fx[k,j,i] = psi1[k,j+1,i] - psi1[k,j,i] + psi2[k+1,j,i] - psi2[k,j,i]  (east face)
      Fy[k,j,i] = -(psi1[k,j+1,i] - psi1[k,j+1,i-1])                          (north face)
      Fz[k,j,i] = -(psi2[k+1,j,i] - psi2[k+1,j,i-1])                          (upper face)
    so every cell's net outflow vanishes and the pole, surface and top faces
    carry none.  psi1 = pe * s_k * cos(theta_face) * g1 and psi2 = pe * s_k *
    cos(theta_j) * g2, with g1, g2 box-filtered N(0,1) fields (as in
    make_problem) and s_k the median longitude coupling of layer k, so the
    transport is a fraction ~pe of the horizontal diffusion on every layer
    and latitude.  Upwinding adds |F| to the coupling of the downstream row:
    F > 0 (towards +i, +j, +k) to txr / tyr / tzr, F < 0 to tx / ty / tz.
    h is unchanged, and with a divergence-free flow it is both the row and
    the column sum of the transport-free part's mass.

    Returns make_problem's dict with tx, ty, tz replaced by the directed
    couplings, txr, tyr, tzr added, and the fluxes fx, fy, fz."""
    P = make_problem(nlon, nlat, nz, sigma, seed, **kw)
    grid = P["grid"]
    rng = np.random.default_rng(seed + 7919)
    g1 = rng.standard_normal((nz, nlat + 1, nlon))
    g2 = rng.standard_normal((nz + 1, nlat, nlon))
    for g in (g1, g2):
        g[:] = box_filter_3pt(g, axis=2, periodic=True)
        g[:] = box_filter_3pt(g, axis=1, periodic=False)
        g[:] = box_filter_3pt(g, axis=0, periodic=False)
    s = np.median(P["tx"].reshape(nz, -1), axis=1)              # [nz]
    cos_f = grid._cos_lat_faces()                               # [nlat+1]
    cos_c = np.cos(grid.lat_centres())                          # [nlat]
    psi1 = pe * s[:, None, None] * cos_f[None, :, None] * g1
    psi1[:, 0, :] = 0.0
    psi1[:, nlat, :] = 0.0
    s2 = np.concatenate([s[:1], s])                             # [nz+1]
    psi2 = pe * s2[:, None, None] * cos_c[None, :, None] * g2
    psi2[0] = 0.0
    psi2[nz] = 0.0
    fx = (psi1[:, 1:, :] - psi1[:, :-1, :]) + (psi2[1:] - psi2[:-1])
    fy = -(psi1[:, 1:, :] - np.roll(psi1[:, 1:, :], 1, axis=2))
    fz = -(psi2[1:] - np.roll(psi2[1:], 1, axis=2))
    fy[:, nlat - 1, :] = 0.0
    fz[nz - 1] = 0.0
    out = dict(P)
    for name, f in (("x", fx), ("y", fy), ("z", fz)):
        t = P["t" + name]
        out["t" + name] = t + np.maximum(-f, 0.0)
        out["t" + name + "r"] = t + np.maximum(f, 0.0)
        out["f" + name] = f
    return out
