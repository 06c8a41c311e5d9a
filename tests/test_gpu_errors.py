"""Failure detection without faulting the GPU: every bad input comes back as
a status code from the C ABI (no trap, no abort), and the handle stays usable."""
import numpy as np
import pytest
import torch

from gpu_common import dev, handle_for, problem

pytestmark = pytest.mark.gpu


def _raises(status, fn):
    from paper_2307_04528_gb300._lib import MGError
    with pytest.raises(MGError) as ei:
        fn()
    assert ei.value.status == status, str(ei.value)


def test_bad_coefficients_rejected_at_setup():
    from paper_2307_04528_gb300 import _lib as L
    P = problem(16, 8, 4)
    for key, where, val in (("h", (0, 0, 0), 0.0), ("h", (1, 2, 3), np.nan),
                            ("tx", (2, 3, 4), -1.0), ("ty", (0, 7, 5), 1.0),  # pole face
                            ("tz", (3, 1, 1), 1.0), ("tz", (1, 1, 1), np.inf)):  # top face
        Q = {k: v.copy() if isinstance(v, np.ndarray) else v for k, v in P.items()}
        Q[key][where] = val
        _raises(L.MG_ERR_COEFF, lambda: handle_for(Q))


def test_nonfinite_rhs_and_nonconvergence_reported():
    from paper_2307_04528_gb300 import _lib as L
    P = problem(32, 16, 8)
    H = handle_for(P, maxit=2)
    b = dev(P["b"])
    b[0, 0, 0] = float("nan")
    _raises(L.MG_ERR_NONFINITE, lambda: H.solve(b))
    _raises(L.MG_ERR_NONFINITE, lambda: H.solve_mixed(b))
    b = dev(P["b"])
    x, info = H.solve(b, tol=1e-12, raise_on_error=False)
    assert info["status"] == L.MG_ERR_NOT_CONVERGED and info["iterations"] == 2
    # the handle is still usable after the failures
    H2 = handle_for(P)
    x, info = H2.solve(b, tol=1e-10)
    assert info["status"] == 0


def test_workspace_and_argument_errors():
    import ctypes
    from paper_2307_04528_gb300 import _lib as L
    lib = L.load()
    P = problem(16, 8, 4)
    co = [dev(P[k]) for k in ("tx", "ty", "tz", "h")]
    g = L.mg_grid(16, 8, 4)
    p = L.default_params()
    need = ctypes.c_size_t()
    assert lib.mg_workspace_bytes(ctypes.byref(g), ctypes.byref(p), ctypes.byref(need)) == 0
    ws = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    c = L.mg_coeffs(*(t.data_ptr() for t in co))
    h = ctypes.c_void_p()
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = lib.mg_setup(ctypes.byref(g), ctypes.byref(c), ctypes.byref(p), ctypes.c_void_p(ws.data_ptr()),
                      need.value - 4096, s, ctypes.byref(h))
    assert st == L.MG_ERR_WORKSPACE and not h.value
    st = lib.mg_setup(ctypes.byref(g), ctypes.byref(c), ctypes.byref(p),
                      ctypes.c_void_p(ws.data_ptr() + 8), need.value - 8, s, ctypes.byref(h))
    assert st == L.MG_ERR_WORKSPACE
    c0 = L.mg_coeffs(0, co[1].data_ptr(), co[2].data_ptr(), co[3].data_ptr())
    st = lib.mg_setup(ctypes.byref(g), ctypes.byref(c0), ctypes.byref(p),
                      ctypes.c_void_p(ws.data_ptr()), need.value, s, ctypes.byref(h))
    assert st == L.MG_ERR_ARG
    H = handle_for(P, mixed=0)
    _raises(L.MG_ERR_ARG, lambda: H.solve_mixed(dev(P["b"])))
    _raises(L.MG_ERR_ARG, lambda: H.level_smooth(99, dev(P["b"])))
    _raises(L.MG_ERR_ARG, lambda: H.level_relax(0, dev(P["b"]), 0))
    _raises(L.MG_ERR_ARG, lambda: H.level_relax(0, dev(P["b"]), 1001))
    _raises(L.MG_ERR_ARG, lambda: H.level_relax(0, dev(P["b"]), 2, prec=L.MG_PREC_FP32))
    b = dev(P["b"])
    assert lib.mg_level_relax(H._hh, 0, 0, 2, ctypes.c_void_p(b.data_ptr()),
                              ctypes.c_void_p(b.data_ptr()), s) == L.MG_ERR_ARG
    last = H.num_levels - 1
    u, bc = torch.zeros_like(b), torch.zeros_like(b)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    assert lib.mg_level_residual_restrict(H._hh, last, 0, ptr(b), ptr(u), ptr(bc), s) == L.MG_ERR_ARG
    assert lib.mg_level_residual_restrict(H._hh, 0, 0, ptr(b), ptr(u), ptr(u), s) == L.MG_ERR_ARG
    assert lib.mg_level_residual_restrict(H._hh, 0, 0, ctypes.c_void_p(b.data_ptr()),
                                          ctypes.c_void_p(b.data_ptr()),
                                          ctypes.c_void_p(b.data_ptr()), s) == L.MG_ERR_ARG
    assert lib.mg_coarse_solve(H._hh, 0, ptr(b), ptr(b), s) == L.MG_ERR_ARG
    _raises(L.MG_ERR_ARG, lambda: handle_for(P, coarse_method=3))

