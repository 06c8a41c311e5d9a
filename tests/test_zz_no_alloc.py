"""The allocation-free residual entry point against the oracle and the
library's own entry points.

mg_residual_norm_noalloc serves callers that cannot allocate device memory
when they need a residual check (a host model owning every device buffer
through its own pool, or C/Fortran host code with no device allocator): it
takes the coefficients directly, needs no handle or workspace, and keeps its
reduction scratch in a static device array.  This file runs last so that a
failure here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest
import torch

from gpu_common import dev, handle_for, host, problem, rel_inf
from oracle import tpmg as O

pytestmark = pytest.mark.gpu


def _call(lib, grid, co, b, x, r):
    rel = ctypes.c_double(-1.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.mg_residual_norm_noalloc(ctypes.byref(grid), ctypes.byref(co),
                                      ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(r.data_ptr()), ctypes.byref(rel), stream)
    return st, rel.value


def _setup(nlon=64, nlat=32, nz=16):
    from paper_2307_04528_gb300 import _lib as L
    P = problem(nlon, nlat, nz, sigma=0.1, seed=42)
    coeffs = [dev(P[k]) for k in ("tx", "ty", "tz", "h")]
    grid = L.mg_grid(nlon, nlat, nz)
    co = L.mg_coeffs(*(t.data_ptr() for t in coeffs))
    return L, L.load(), P, coeffs, grid, co


def test_noalloc_residual_matches_oracle_and_handle_twice():
    """Two calls in a row, nothing carried over.  A random iterate (terms of
    the residual without cancellation) against the oracle; a converged one
    (the residual a ~1e-9 difference of terms up to ~1e6 larger, so only the
    same operation order reproduces it to rounding) against the handle's
    residual entry point."""
    L, lib, P, coeffs, grid, co = _setup()
    H = handle_for(P, mixed=0)
    fine = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], O.MGParams(levels=1))[0]
    b = dev(P["b"])
    r = torch.empty_like(b)
    xr = np.random.default_rng(3).standard_normal(P["b"].shape)
    x, info = H.solve(b, tol=1e-9)
    for xx in (dev(xr), x):
        st, rel = _call(lib, grid, co, b, xx, r)
        assert st == 0, lib.mg_last_error()
        torch.cuda.synchronize()
        r_ref = H.level_residual(0, b, xx)
        assert rel_inf(host(r), host(r_ref)) <= 1e-13
        rel_ref = float(torch.linalg.vector_norm(r_ref) / torch.linalg.vector_norm(b))
        assert abs(rel - rel_ref) <= 1e-12 * rel_ref
        if xx is not x:
            r_orc = O.residual(fine, P["b"], xr)
            assert rel_inf(host(r), r_orc) <= 1e-13
            rel_orc = O.norm2(r_orc) / O.norm2(P["b"])
            assert abs(rel - rel_orc) <= 1e-12 * rel_orc
        else:
            assert abs(rel - info["rel_res"]) <= 1e-12 * info["rel_res"]


def test_noalloc_allocates_no_device_memory():
    L, lib, P, coeffs, grid, co = _setup()
    b = dev(P["b"])
    x = torch.zeros_like(b)
    r = torch.empty_like(b)
    assert _call(lib, grid, co, b, x, r)[0] == 0  # first call: the array's address is looked up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        st, rel = _call(lib, grid, co, b, x, r)
        assert st == 0 and rel == pytest.approx(1.0, abs=1e-15)  # x = 0: r = b
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_noalloc_rejects_nonfinite_norms():
    L, lib, P, coeffs, grid, co = _setup()
    x = torch.zeros(P["b"].shape, dtype=torch.float64, device="cuda")
    r = torch.empty_like(x)
    for bad in (np.inf, np.nan):
        bh = P["b"].copy()
        bh[3, 5, 7] = bad
        st, rel = _call(lib, grid, co, dev(bh), x, r)
        assert st == L.MG_ERR_NONFINITE, (bad, st)
        assert rel == -1.0  # left untouched
    b = dev(P["b"])
    bh = P["b"].copy()
    bh[0, 0, 0] = 1e300  # b finite, but the squared norms overflow to Inf
    st, _ = _call(lib, grid, co, dev(bh), x, r)
    assert st == L.MG_ERR_NONFINITE
    st, rel = _call(lib, grid, co, b, x, r)  # the entry point stays usable
    assert st == 0 and rel == pytest.approx(1.0, abs=1e-15)


def test_noalloc_rejects_grids_beyond_its_static_scratch():
    from paper_2307_04528_gb300 import _lib as L
    lib = L.load()
    grid = L.mg_grid(4096, 1024, 1)    # 4,194,304 columns > 2,097,152
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    co = L.mg_coeffs(*(one.data_ptr(),) * 4)
    st, _ = _call(lib, grid, co, one, one, one)
    assert st == L.MG_ERR_ARG
    assert b"static scratch limit" in lib.mg_last_error()
