"""The allocation-free residual entry point against the library's own ones.

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

pytestmark = pytest.mark.gpu


def _call(lib, L, grid, co, b, x):
    r = torch.empty_like(b)
    rel = ctypes.c_double(-1.0)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.mg_residual_norm_noalloc(ctypes.byref(grid), ctypes.byref(co),
                                      ctypes.c_void_p(b.data_ptr()), ctypes.c_void_p(x.data_ptr()),
                                      ctypes.c_void_p(r.data_ptr()), ctypes.byref(rel), stream)
    return st, r, rel.value


def test_noalloc_residual_matches_handle_entry_points_twice():
    from paper_2307_04528_gb300 import _lib as L
    lib = L.load()
    nlon, nlat, nz = 64, 32, 16
    P = problem(nlon, nlat, nz, sigma=0.1, seed=42)
    coeffs = [dev(P[k]) for k in ("tx", "ty", "tz", "h")]
    H = handle_for(P, mixed=0)
    b = dev(P["b"])
    grid = L.mg_grid(nlon, nlat, nz)
    co = L.mg_coeffs(*(t.data_ptr() for t in coeffs))
    # two calls in a row with different iterates: nothing may carry over
    for tol in (1e-4, 1e-9):
        x, info = H.solve(b, tol=tol)
        st, r, rel = _call(lib, L, grid, co, b, x)
        assert st == 0, lib.mg_last_error()
        r_ref = H.level_residual(0, b, x)
        torch.cuda.synchronize()
        assert rel_inf(host(r), host(r_ref)) <= 1e-13
        assert abs(rel - info["rel_res"]) <= 1e-12 * info["rel_res"]


def test_noalloc_rejects_grids_beyond_its_static_scratch():
    from paper_2307_04528_gb300 import _lib as L
    lib = L.load()
    grid = L.mg_grid(4096, 1024, 1)    # 4,194,304 columns > 2,097,152
    one = torch.zeros(1, dtype=torch.float64, device="cuda")
    co = L.mg_coeffs(*(one.data_ptr(),) * 4)
    st, _, _ = _call(lib, L, grid, co, one, one)
    assert st == L.MG_ERR_ARG
    assert b"static scratch limit" in lib.mg_last_error()
