"""Python face of libtpmg: a handle over the C ABI and the differentiable solve.

Torch provides device memory (the workspace and the fields) and the current
CUDA stream; every numerical step runs in libtpmg's kernels.
"""
from __future__ import annotations

import ctypes
import warnings

import torch

from . import _lib as L


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _field(t, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
        raise ValueError(f"{name}: need contiguous {dtype} {tuple(shape)}, got "
                         f"{t.dtype} {tuple(t.shape)}")
    return t


class MGHandle:
    """Multigrid hierarchy for H u = b on an [nz, nlat, nlon] lat-lon grid.

    tx, ty, tz, h: CUDA float64 tensors (copied into the workspace at setup).
    params: keyword overrides of mg_params (levels, nu1, nu2, coarse_iters,
    method, mixed, maxit, inner_maxit, omega, alpha_c, inner_tol,
    coarse_method, line_sweeps).
    """

    @classmethod
    def borrow(cls, ptr, shape, device, owner):
        """Wrap a handle owned by `owner` (e.g. one system of an MGBatch)."""
        self = cls.__new__(cls)
        self.lib = L.load()
        self.shape = tuple(shape)
        self.device = device
        self._h = None          # not ours to destroy
        self._borrowed = ctypes.c_void_p(ptr)
        self._owner = owner
        return self

    @property
    def _hh(self):
        return self._h if self._h is not None else self._borrowed

    def __init__(self, tx, ty, tz, h, stream=None, **params):
        self.lib = L.load()
        nz, nlat, nlon = h.shape
        self.shape = (nz, nlat, nlon)
        for name, t in (("tx", tx), ("ty", ty), ("tz", tz), ("h", h)):
            _field(t, torch.float64, self.shape, name)
        self.device = h.device
        self.grid = L.mg_grid(nlon, nlat, nz)
        self.params = L.default_params(**params)
        nbytes = ctypes.c_size_t(0)
        L.check(self.lib.mg_workspace_bytes(ctypes.byref(self.grid), ctypes.byref(self.params),
                                            ctypes.byref(nbytes)))
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        co = L.mg_coeffs(tx.data_ptr(), ty.data_ptr(), tz.data_ptr(), h.data_ptr())
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            L.check(self.lib.mg_setup(ctypes.byref(self.grid), ctypes.byref(co),
                                      ctypes.byref(self.params), _ptr(self.workspace),
                                      nbytes, _stream(stream), ctypes.byref(self._h)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self.lib.mg_destroy(h)
            self._h = None

    # ------------------------------------------------------------- queries
    @property
    def num_levels(self) -> int:
        return int(self.lib.mg_num_levels(self._hh))

    def level_shape(self, level: int):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        L.check(self.lib.mg_level_shape(self._hh, level, ctypes.byref(a), ctypes.byref(b),
                                        ctypes.byref(c)))
        return (c.value, b.value, a.value)

    def level_coeffs(self, level: int):
        shp = self.level_shape(level)
        out = [torch.empty(shp, dtype=torch.float64, device=self.device) for _ in range(4)]
        L.check(self.lib.mg_level_coeffs(self._hh, level, *map(_ptr, out), _stream()))
        return out

    @property
    def fp32_scale(self) -> float:
        return float(self.lib.mg_fp32_scale(self._hh))

    # ------------------------------------------------------------- fine level
    def apply(self, x, y=None):
        _field(x, torch.float64, self.shape, "x")
        y = torch.empty_like(x) if y is None else y
        L.check(self.lib.mg_apply(self._hh, _ptr(x), _ptr(y), _stream()))
        return y

    def vcycle(self, r, e=None, prec=L.MG_PREC_FP64):
        """e = V r, one V-cycle from zero; prec MG_PREC_FP32 runs the FP32
        hierarchy (scaled coefficients, see fp32_scale) on float32 r."""
        _field(r, self._dt(prec), self.shape, "r")
        e = torch.empty_like(r) if e is None else e
        if prec == L.MG_PREC_FP64:
            L.check(self.lib.mg_vcycle(self._hh, _ptr(r), _ptr(e), _stream()))
        else:
            L.check(self.lib.mg_vcycle_prec(self._hh, prec, _ptr(r), _ptr(e), _stream()))
        return e

    def _solve(self, fn, b, x, tol, history_cap, raise_on):
        _field(b, torch.float64, self.shape, "b")
        x = torch.zeros_like(b) if x is None else x
        _field(x, torch.float64, self.shape, "x")
        hist = (ctypes.c_double * history_cap)()
        st = L.mg_stats(0, 0, 0.0, hist, history_cap, 0)
        status = fn(self._hh, _ptr(b), _ptr(x), float(tol), ctypes.byref(st), _stream())
        if raise_on:
            L.check(status)
        info = dict(status=status, iterations=st.iterations, inner_iterations=st.inner_iterations,
                    rel_res=st.rel_res, history=[hist[i] for i in range(st.history_len)])
        return x, info

    def solve(self, b, x=None, tol=1e-10, history_cap=512, raise_on_error=True):
        """FP64 multigrid solve; x is the initial guess and is overwritten."""
        return self._solve(self.lib.mg_solve, b, x, tol, history_cap, raise_on_error)

    def solve_mixed(self, b, x=None, tol=1e-10, history_cap=512, raise_on_error=True):
        """FP32 multigrid inside FP64 refinement (needs mixed=1 at setup)."""
        return self._solve(self.lib.mg_solve_mixed, b, x, tol, history_cap, raise_on_error)

    def solve_single(self, b, x=None, tol=1e-6, history_cap=4096, raise_on_error=True):
        """The whole solve in FP32 (float32 b and x; needs mixed=1 at setup),
        with the configured method; x is the initial guess, overwritten."""
        _field(b, torch.float32, self.shape, "b")
        x = torch.zeros_like(b) if x is None else x
        _field(x, torch.float32, self.shape, "x")
        hist = (ctypes.c_double * history_cap)()
        st = L.mg_stats(0, 0, 0.0, hist, history_cap, 0)
        status = self.lib.mg_solve_single(self._hh, _ptr(b), _ptr(x), float(tol),
                                          ctypes.byref(st), _stream())
        if raise_on_error:
            L.check(status)
        info = dict(status=status, iterations=st.iterations, rel_res=st.rel_res,
                    history=[hist[i] for i in range(st.history_len)])
        return x, info

    def coeff_grad(self, lam, x):
        outs = [torch.empty_like(x) for _ in range(4)]
        L.check(self.lib.mg_coeff_grad(self._hh, _ptr(lam), _ptr(x), *map(_ptr, outs), _stream()))
        return tuple(outs)  # gh, gtx, gty, gtz

    # ------------------------------------------------------------- measurement
    def profile(self, on=True):
        """on: False/0 off, True/1 fine-level launches, 2 every level."""
        L.check(self.lib.mg_profile_enable(self._hh, int(on)))

    def profile_read(self, kind: int, level: int, prec: int):
        n, ms = ctypes.c_int(0), ctypes.c_double(0.0)
        L.check(self.lib.mg_profile_read(self._hh, kind, level, prec, ctypes.byref(n),
                                         ctypes.byref(ms)))
        return n.value, ms.value

    # ------------------------------------------------------------- per level
    def _dt(self, prec):
        return torch.float64 if prec == L.MG_PREC_FP64 else torch.float32

    def level_apply(self, level, x, prec=L.MG_PREC_FP64):
        y = torch.empty_like(x)
        L.check(self.lib.mg_level_apply(self._hh, level, prec, _ptr(x), _ptr(y), _stream()))
        return y

    def level_residual(self, level, b, u, prec=L.MG_PREC_FP64):
        r = torch.empty_like(b)
        L.check(self.lib.mg_level_residual(self._hh, level, prec, _ptr(b), _ptr(u), _ptr(r),
                                           _stream()))
        return r

    def level_smooth(self, level, b, u_in=None, prec=L.MG_PREC_FP64):
        out = torch.empty_like(b)
        L.check(self.lib.mg_level_smooth(self._hh, level, prec, _ptr(b), _ptr(u_in), _ptr(out),
                                         _stream()))
        return out

    def level_residual_restrict(self, level, b, u, prec=L.MG_PREC_FP64):
        """R (b - H u) on level -> level + 1 in one pass."""
        shp = self.level_shape(level + 1)
        bc = torch.empty(shp, dtype=b.dtype, device=b.device)
        L.check(self.lib.mg_level_residual_restrict(self._hh, level, prec, _ptr(b), _ptr(u),
                                                    _ptr(bc), _stream()))
        return bc

    def level_presmooth_restrict(self, level, b, u, prec=L.MG_PREC_FP64):
        """R ((1 - omega) b + horizontal couplings of u): the restricted residual
        after the sweep from zero u = omega H_z^{-1} b."""
        shp = self.level_shape(level + 1)
        bc = torch.empty(shp, dtype=b.dtype, device=b.device)
        L.check(self.lib.mg_level_presmooth_restrict(self._hh, level, prec, _ptr(b), _ptr(u),
                                                     _ptr(bc), _stream()))
        return bc

    def coarse_solve(self, b, prec=L.MG_PREC_FP64):
        """The V-cycle's coarsest-level solve (block-Jacobi sweeps or PCG, as
        configured) applied to b on the coarsest level."""
        out = torch.empty_like(b)
        L.check(self.lib.mg_coarse_solve(self._hh, prec, _ptr(b), _ptr(out), _stream()))
        return out

    def level_relax(self, level, b, sweeps, prec=L.MG_PREC_FP64):
        """`sweeps` sweeps from the zero guess (on the coarsest level with
        sweeps = coarse_iters: the V-cycle's coarsest-level solve)."""
        out = torch.empty_like(b)
        L.check(self.lib.mg_level_relax(self._hh, level, prec, int(sweeps), _ptr(b), _ptr(out),
                                        _stream()))
        return out

    def level_smooth_dot(self, level, b, u_in, prec=L.MG_PREC_FP64):
        """One sweep plus <b, u_out> (the V-cycle's last sweep with the CG
        inner product fused in)."""
        out = torch.empty_like(b)
        dot = ctypes.c_double()
        L.check(self.lib.mg_level_smooth_dot(self._hh, level, prec, _ptr(b), _ptr(u_in), _ptr(out),
                                             ctypes.byref(dot), _stream()))
        return out, dot.value

    def level_dir_apply(self, level, z, d_old=None, beta=0.0, prec=L.MG_PREC_FP64):
        """The fused CG step: d_new = z + beta d_old (d_old None: z), q = H d_new,
        and <d_new, q>.  Returns (d_new, q, dot)."""
        d_new, q = torch.empty_like(z), torch.empty_like(z)
        dot = ctypes.c_double()
        L.check(self.lib.mg_level_dir_apply(self._hh, level, prec, _ptr(z), _ptr(d_old),
                                            float(beta), _ptr(d_new), _ptr(q), ctypes.byref(dot),
                                            _stream()))
        return d_new, q, dot.value

    def level_restrict(self, level, r, prec=L.MG_PREC_FP64):
        shp = self.level_shape(level + 1)
        bc = torch.empty(shp, dtype=r.dtype, device=r.device)
        L.check(self.lib.mg_level_restrict(self._hh, level, prec, _ptr(r), _ptr(bc), _stream()))
        return bc

    def level_prolong_add(self, level, ec, u, prec=L.MG_PREC_FP64):
        L.check(self.lib.mg_level_prolong_add(self._hh, level, prec, _ptr(ec), _ptr(u), _stream()))
        return u


def cast_fp32(x, scale):
    """The FP32 rounding of x * scale (mg_cast_fp32; x a CUDA float64
    tensor): the right-hand side handed to an FP32 inner solve."""
    if x.dtype != torch.float64 or not x.is_cuda:
        raise TypeError("x must be a CUDA float64 tensor")
    x = x.contiguous()
    y = torch.empty(x.shape, dtype=torch.float32, device=x.device)
    L.check(L.load().mg_cast_fp32(_ptr(x), _ptr(y), float(scale), x.numel(), _stream()))
    return y


def update_fp64(x, e, scale):
    """x += scale * e in FP64 in place (mg_update_fp64; x CUDA float64, e
    CUDA float32 of the same size): the refinement's update."""
    if x.dtype != torch.float64 or e.dtype != torch.float32 or not (x.is_cuda and e.is_cuda):
        raise TypeError("x must be CUDA float64 and e CUDA float32")
    if x.numel() != e.numel() or not x.is_contiguous():
        raise ValueError("x must be contiguous and e of the same size")
    e = e.contiguous()
    L.check(L.load().mg_update_fp64(_ptr(x), _ptr(e), float(scale), x.numel(), _stream()))
    return x


class MGFloorWarning(RuntimeWarning):
    """A differentiable solve stopped on maxit above its tolerance but below the
    caller's floor_accept, and its solution was used."""


def _solve_checked(handle, b, tol, floor_accept=None, mixed=False, **solve_kw):
    """Solve and raise on any failure, except that a solve stopping on maxit
    with rel_res <= floor_accept is accepted with an MGFloorWarning.  The
    FP64 rounding floor of the residual (rounding of x times the vertical
    couplings: ~1e-12..1e-10 relative, higher for smooth right-hand sides
    such as an adjoint dL/dx) can sit above a tight tol while the solution
    is accurate; floor_accept=None (the default) accepts nothing.  mixed: FP32
    multigrid inside FP64 refinement (the handle needs mixed=1)."""
    fn = handle.solve_mixed if mixed else handle.solve
    x, info = fn(b, tol=tol, raise_on_error=False, **solve_kw)
    st = info["status"]
    if st == L.MG_OK:
        return x, info
    if (st == L.MG_ERR_NOT_CONVERGED and floor_accept is not None
            and info["rel_res"] <= floor_accept):
        warnings.warn(MGFloorWarning(
            f"solve stopped after {info['iterations']} iterations at relative residual "
            f"{info['rel_res']:.3e} > tol {tol:.1e}; accepted (floor_accept {floor_accept:.1e})"),
            stacklevel=3)
        return x, info
    L.check(st)
    return x, info


class MGBatch:
    """Ensemble of independent systems of uneven sizes solved together.

    systems: list of (tx, ty, tz, h) CUDA float64 tensors, one tuple per
    system.  params: keyword overrides of mg_params (common to all)."""

    def __init__(self, systems, stream=None, **params):
        self.lib = L.load()
        self.n = len(systems)
        self.shapes = []
        grids = (L.mg_grid * self.n)()
        coeffs = (L.mg_coeffs * self.n)()
        for i, (tx, ty, tz, h) in enumerate(systems):
            shp = tuple(h.shape)
            for name, t in (("tx", tx), ("ty", ty), ("tz", tz), ("h", h)):
                _field(t, torch.float64, shp, name)
            self.shapes.append(shp)
            grids[i] = L.mg_grid(shp[2], shp[1], shp[0])
            coeffs[i] = L.mg_coeffs(tx.data_ptr(), ty.data_ptr(), tz.data_ptr(), h.data_ptr())
        self.device = systems[0][3].device
        self.params = L.default_params(**params)
        nbytes = ctypes.c_size_t(0)
        L.check(self.lib.mg_batch_workspace_bytes(self.n, grids, ctypes.byref(self.params),
                                                  ctypes.byref(nbytes)))
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        self._b = ctypes.c_void_p()
        L.check(self.lib.mg_batch_setup(self.n, grids, coeffs, ctypes.byref(self.params),
                                        _ptr(self.workspace), nbytes, _stream(stream),
                                        ctypes.byref(self._b)))

    def __del__(self):
        b = getattr(self, "_b", None)
        if b is not None and b.value:
            self.lib.mg_batch_destroy(b)
            self._b = None

    def handle(self, i):
        """The handle of system i (for single-system calls on the same data)."""
        out = ctypes.c_void_p()
        L.check(self.lib.mg_batch_handle(self._b, i, ctypes.byref(out)))
        return MGHandle.borrow(out.value, self.shapes[i], self.device, self)

    def tuning(self):
        v = [ctypes.c_int() for _ in range(4)]
        L.check(self.lib.mg_batch_tuning(self._b, *map(ctypes.byref, v)))
        return dict(zip(("smooth_block", "smooth_grid", "cell_grid", "vec_grid"),
                        (x.value for x in v)))

    def solve(self, bs, xs=None, tol=1e-8, mixed=True, raise_on_error=True):
        """Solve every system; bs, xs: lists of CUDA float64 tensors (xs is
        the initial guess, overwritten).  Returns (xs, per-system infos)."""
        if xs is None:
            xs = [torch.zeros_like(b) for b in bs]
        for i, (b, x) in enumerate(zip(bs, xs)):
            _field(b, torch.float64, self.shapes[i], f"b[{i}]")
            _field(x, torch.float64, self.shapes[i], f"x[{i}]")
        bp = (ctypes.c_void_p * self.n)(*(b.data_ptr() for b in bs))
        xp = (ctypes.c_void_p * self.n)(*(x.data_ptr() for x in xs))
        stats = (L.mg_stats * self.n)()
        status = (ctypes.c_int * self.n)()
        st = self.lib.mg_batch_solve(self._b, bp, xp, float(tol), int(bool(mixed)), stats,
                                     status, _stream())
        if raise_on_error:
            L.check(st)
        infos = [dict(status=status[i], iterations=stats[i].iterations,
                      inner_iterations=stats[i].inner_iterations, rel_res=stats[i].rel_res)
                 for i in range(self.n)]
        return xs, infos


class MGSolveFn(torch.autograd.Function):
    """x = H(h, tx, ty, tz)^{-1} b as a differentiable function.

    Backward solves the adjoint system H^T lambda = dL/dx with the same
    hierarchy (H is symmetric: each face couples its two cells with one
    coefficient, so the transposed stencil is the stencil) and forms the
    coefficient gradient with one fused kernel; only the solution x is kept
    from the forward pass, no iterate.  Both solves must reach tol; with
    floor_accept set, a solve that stops on maxit at or below that relative
    residual is used with an MGFloorWarning.  The statuses of the two solves
    are kept in ctx.infos (forward, then adjoint)."""

    @staticmethod
    def forward(ctx, b, h, tx, ty, tz, tol=1e-11, params=None, floor_accept=None, mixed=False):
        params = dict(params or {})
        if mixed:
            params["mixed"] = 1
        handle = MGHandle(tx.detach().contiguous(), ty.detach().contiguous(),
                          tz.detach().contiguous(), h.detach().contiguous(), **params)
        x, info = _solve_checked(handle, b.detach().contiguous(), tol, floor_accept, mixed)
        ctx.handle = handle
        ctx.tol = tol
        ctx.floor_accept = floor_accept
        ctx.mixed = mixed
        ctx.infos = [info]
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        lam, info = _solve_checked(ctx.handle, gx.contiguous(), ctx.tol, ctx.floor_accept,
                                   ctx.mixed)
        ctx.infos.append(info)
        gh, gtx, gty, gtz = ctx.handle.coeff_grad(lam, x)
        return lam, gh, gtx, gty, gtz, None, None, None, None


def mg_solve_fn(b, h, tx, ty, tz, tol=1e-11, floor_accept=None, mixed=False, **params):
    """Differentiable solve (MGSolveFn); params: mg_params overrides; mixed:
    both solves with FP32 multigrid inside FP64 refinement."""
    return MGSolveFn.apply(b, h, tx, ty, tz, tol, params, floor_accept, mixed)


_NS_ARRAYS = ("h", "tx", "ty", "tz", "txr", "tyr", "tzr")


class NSHandle:
    """Multigrid hierarchies of a nonsymmetric operator H (directed couplings,
    mg_ns_* in include/tpmg.h) and of its transpose.

    h, tx, ty, tz, txr, tyr, tzr: CUDA float64 tensors [nz, nlat, nlon]
    (tx[c]: row c's coupling to its east neighbour; txr[c]: that neighbour's
    row's coupling back to c; likewise north and up; h: the row sums).
    params: mg_params overrides; method MG_METHOD_BICGSTAB (default here) or
    MG_METHOD_STATIONARY.  Every call takes transpose=False (H) or True (H^T).
    """

    def __init__(self, h, tx, ty, tz, txr, tyr, tzr, stream=None, **params):
        self.lib = L.load()
        nz, nlat, nlon = h.shape
        self.shape = (nz, nlat, nlon)
        arrays = (h, tx, ty, tz, txr, tyr, tzr)
        for name, t in zip(_NS_ARRAYS, arrays):
            _field(t, torch.float64, self.shape, name)
        self.device = h.device
        self.grid = L.mg_grid(nlon, nlat, nz)
        params.setdefault("method", L.MG_METHOD_BICGSTAB)
        self.params = L.default_params(**params)
        nbytes = ctypes.c_size_t(0)
        L.check(self.lib.mg_ns_workspace_bytes(ctypes.byref(self.grid),
                                               ctypes.byref(self.params), ctypes.byref(nbytes)))
        self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        co = L.mg_ns_coeffs(*(t.data_ptr() for t in arrays))
        self._h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            L.check(self.lib.mg_ns_setup(ctypes.byref(self.grid), ctypes.byref(co),
                                         ctypes.byref(self.params), _ptr(self.workspace),
                                         nbytes, _stream(stream), ctypes.byref(self._h)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            self.lib.mg_ns_destroy(h)
            self._h = None

    @property
    def num_levels(self) -> int:
        return int(self.lib.mg_ns_num_levels(self._h))

    def level_shape(self, level: int):
        a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        L.check(self.lib.mg_ns_level_shape(self._h, level, ctypes.byref(a), ctypes.byref(b),
                                           ctypes.byref(c)))
        return (c.value, b.value, a.value)

    def level_coeffs(self, level: int, transpose=False):
        """The level's (h, tx, ty, tz, txr, tyr, tzr) of H, or of H^T."""
        shp = self.level_shape(level)
        out = [torch.empty(shp, dtype=torch.float64, device=self.device) for _ in range(7)]
        L.check(self.lib.mg_ns_level_coeffs(self._h, level, int(transpose), *map(_ptr, out),
                                            _stream()))
        return out

    def apply(self, x, transpose=False, y=None):
        _field(x, torch.float64, self.shape, "x")
        y = torch.empty_like(x) if y is None else y
        L.check(self.lib.mg_ns_apply(self._h, int(transpose), _ptr(x), _ptr(y), _stream()))
        return y

    @property
    def fp32_scale(self) -> float:
        return float(self.lib.mg_ns_fp32_scale(self._h))

    def vcycle(self, r, transpose=False, e=None, prec=L.MG_PREC_FP64):
        """e = V r of H (or H^T); prec MG_PREC_FP32 runs the FP32 hierarchy
        (scaled arrays, see fp32_scale) on float32 r."""
        dt = torch.float64 if prec == L.MG_PREC_FP64 else torch.float32
        _field(r, dt, self.shape, "r")
        e = torch.empty_like(r) if e is None else e
        L.check(self.lib.mg_ns_vcycle_prec(self._h, int(transpose), prec, _ptr(r), _ptr(e),
                                           _stream()))
        return e

    def level_smooth(self, level, b, u_in=None, transpose=False, prec=L.MG_PREC_FP64):
        """One sweep of Eq. (1) on a level of H (or H^T); u_in None: zero guess."""
        out = torch.empty_like(b)
        L.check(self.lib.mg_ns_level_smooth(self._h, level, int(transpose), prec, _ptr(b),
                                            _ptr(u_in), _ptr(out), _stream()))
        return out

    def _solve(self, fn, b, x, tol, transpose, history_cap, raise_on):
        _field(b, torch.float64, self.shape, "b")
        x = torch.zeros_like(b) if x is None else x
        _field(x, torch.float64, self.shape, "x")
        hist = (ctypes.c_double * history_cap)()
        st = L.mg_stats(0, 0, 0.0, hist, history_cap, 0)
        status = fn(self._h, int(transpose), _ptr(b), _ptr(x), float(tol), ctypes.byref(st),
                    _stream())
        if raise_on:
            L.check(status)
        info = dict(status=status, iterations=st.iterations, inner_iterations=st.inner_iterations,
                    rel_res=st.rel_res, history=[hist[i] for i in range(st.history_len)])
        return x, info

    def solve(self, b, x=None, tol=1e-10, transpose=False, history_cap=512,
              raise_on_error=True):
        """Solve H x = b (or H^T x = b) in FP64; x is the initial guess, overwritten."""
        return self._solve(self.lib.mg_ns_solve, b, x, tol, transpose, history_cap,
                           raise_on_error)

    def solve_mixed(self, b, x=None, tol=1e-10, transpose=False, history_cap=512,
                    raise_on_error=True):
        """The same solve with FP32 multigrid inside FP64 refinement (mixed=1)."""
        return self._solve(self.lib.mg_ns_solve_mixed, b, x, tol, transpose, history_cap,
                           raise_on_error)

    def coeff_grad(self, lam, x):
        """(gh, gtx, gty, gtz, gtxr, gtyr, gtzr) = -lam^T (dH/dtheta) x."""
        out = [torch.empty_like(x) for _ in range(7)]
        L.check(self.lib.mg_ns_coeff_grad(self._h, _ptr(lam), _ptr(x), *map(_ptr, out),
                                          _stream()))
        return out


class NSSolveFn(torch.autograd.Function):
    """x = H^{-1} b for the nonsymmetric operator, differentiable in b and the
    seven arrays.  Backward solves the adjoint system H^T lambda = dL/dx on
    the transposed hierarchy (a different operator from H now) and forms
    the seven gradients in one kernel; statuses in ctx.infos."""

    @staticmethod
    def forward(ctx, b, h, tx, ty, tz, txr, tyr, tzr, tol=1e-10, params=None,
                floor_accept=None, mixed=False):
        arrays = [t.detach().contiguous() for t in (h, tx, ty, tz, txr, tyr, tzr)]
        params = dict(params or {})
        if mixed:
            params["mixed"] = 1
        handle = NSHandle(*arrays, **params)
        x, info = _solve_checked(handle, b.detach().contiguous(), tol, floor_accept, mixed)
        ctx.handle, ctx.tol, ctx.floor_accept, ctx.infos = handle, tol, floor_accept, [info]
        ctx.mixed = mixed
        ctx.save_for_backward(x)
        return x

    @staticmethod
    def backward(ctx, gx):
        (x,) = ctx.saved_tensors
        lam, info = _solve_checked(ctx.handle, gx.contiguous(), ctx.tol, ctx.floor_accept,
                                   ctx.mixed, transpose=True)
        ctx.infos.append(info)
        grads = ctx.handle.coeff_grad(lam, x)
        return (lam, *grads, None, None, None, None)


def ns_solve_fn(b, h, tx, ty, tz, txr, tyr, tzr, tol=1e-10, floor_accept=None, mixed=False,
                **params):
    """Differentiable nonsymmetric solve (NSSolveFn); params: mg_params
    overrides; mixed: both solves with FP32 multigrid inside FP64 refinement."""
    return NSSolveFn.apply(b, h, tx, ty, tz, txr, tyr, tzr, tol, params, floor_accept, mixed)
