"""GPU parity of the nonsymmetric operator (mg_ns_*) against its oracle
(oracle/ns.py) on the same seeded inputs: both hierarchies, the apply and the
transposed-stencil apply, every level's sweep of H and of H^T, the V-cycles,
the solves of H and H^T, the gradient and the differentiable solve; the
symmetric case against the symmetric handle; properties at the operational
size."""
import numpy as np
import pytest
import torch

from gpu_common import dev, host, rel_2, rel_inf
from oracle import ns as N
from oracle import tpmg as O
from synthetic import make_ns_problem, make_problem

pytestmark = pytest.mark.gpu

NAMES = ("h", "tx", "ty", "tz", "txr", "tyr", "tzr")


def _ns_problem(nlon, nlat, nz, seed=21, pe=0.3, sigma=0.2):
    return make_ns_problem(nlon, nlat, nz, sigma, seed, pe=pe)


def _handle(P, **params):
    from paper_2307_04528_gb300.solver import NSHandle
    return NSHandle(*(dev(P[k]) for k in NAMES), **params)


def _oracle(P, **params):
    p = O.MGParams(**params)
    L = N.build_hierarchy(*(P[k] for k in NAMES), p)
    return L, N.transposed(L), p


# 96 x 46: 4416 columns, 34.5 blocks of 128 (ragged), five levels
SHAPES = [(96, 46, 12), (64, 32, 16)]


@pytest.mark.parametrize("shape", SHAPES)
def test_both_hierarchies_match_the_oracle(shape):
    P = _ns_problem(*shape)
    H = _handle(P)
    L, T, _ = _oracle(P)
    assert H.num_levels == len(L)
    for l in range(len(L)):
        for tr, lev in ((False, L[l]), (True, T[l])):
            got = H.level_coeffs(l, transpose=tr)
            want = lev.arrays()
            for name, g, w in zip(NAMES, got, want):
                assert host(g).shape == w.shape
                assert rel_inf(host(g), w) <= 1e-15, (l, tr, name)


@pytest.mark.parametrize("shape", SHAPES)
def test_apply_and_transposed_apply(shape):
    P = _ns_problem(*shape)
    H = _handle(P)
    L, T, _ = _oracle(P)
    x = np.random.default_rng(1).standard_normal(P["h"].shape)
    xd = dev(x)
    assert rel_inf(host(H.apply(xd)), N.apply(L[0], x)) <= 1e-13
    assert rel_inf(host(H.apply(xd, transpose=True)), N.apply(T[0], x)) <= 1e-13
    # <H x, y> = <x, H^T y>
    y = dev(np.random.default_rng(2).standard_normal(P["h"].shape))
    a = float(torch.dot(H.apply(xd).ravel(), y.ravel()))
    b = float(torch.dot(xd.ravel(), H.apply(y, transpose=True).ravel()))
    assert abs(a - b) <= 1e-12 * float(torch.linalg.vector_norm(H.apply(xd)) *
                                       torch.linalg.vector_norm(y))


@pytest.mark.parametrize("transpose", [False, True])
def test_sweeps_on_every_level(transpose):
    P = _ns_problem(96, 46, 12)
    H = _handle(P)
    L, T, p = _oracle(P)
    levs = T if transpose else L
    rng = np.random.default_rng(3)
    for l, lev in enumerate(levs):
        b = rng.standard_normal(lev.shape)
        u = rng.standard_normal(lev.shape)
        z = H.level_smooth(l, dev(b), None, transpose=transpose)
        assert rel_inf(host(z), N.smooth_from_zero(lev, b, p.omega)) <= 1e-12, (l, "zero")
        s = H.level_smooth(l, dev(b), dev(u), transpose=transpose)
        assert rel_inf(host(s), N.smooth(lev, b, u, p.omega)) <= 1e-12, (l, "guess")


@pytest.mark.parametrize("params", [{}, {"nu1": 2, "nu2": 2}, {"nu1": 2, "nu2": 1},
                                    {"coarse_iters": 5}])
def test_vcycles_of_h_and_its_transpose(params):
    P = _ns_problem(96, 46, 12)
    H = _handle(P, **params)
    L, T, p = _oracle(P, **params)
    r = np.random.default_rng(4).standard_normal(P["h"].shape)
    for tr, levs in ((False, L), (True, T)):
        e = host(H.vcycle(dev(r), transpose=tr))
        assert rel_inf(e, N.vcycle(levs, r, p)) <= 1e-11, (tr, params)


@pytest.mark.parametrize("method", ["stationary", "bicgstab"])
@pytest.mark.parametrize("transpose", [False, True])
def test_solves_match_the_oracle(method, transpose):
    from paper_2307_04528_gb300 import _lib as L_
    P = _ns_problem(64, 32, 16)
    code = L_.MG_METHOD_STATIONARY if method == "stationary" else L_.MG_METHOD_BICGSTAB
    H = _handle(P, method=code)
    L, T, _ = _oracle(P)
    x, info = H.solve(dev(P["b"]), tol=1e-10, transpose=transpose)
    xo, hist, st = N.solve(T if transpose else L, P["b"], 1e-10, O.MGParams(method=method))
    assert st == N.OK and info["status"] == 0
    assert info["rel_res"] <= 1e-10
    assert rel_2(host(x), xo) <= 1e-8
    assert abs(info["iterations"] - (len(hist) - 1)) <= 2
    # the library's reported residual is the oracle's residual of the GPU solution
    A = T[0] if transpose else L[0]
    true = np.linalg.norm(N.residual(A, P["b"], host(x))) / np.linalg.norm(P["b"])
    assert true <= 1.5e-10


def test_symmetric_case_equals_the_symmetric_handle():
    from paper_2307_04528_gb300.solver import MGHandle
    P = make_problem(96, 46, 12, 0.2, 22)
    c = {"h": P["h"], "tx": P["tx"], "ty": P["ty"], "tz": P["tz"],
         "txr": P["tx"], "tyr": P["ty"], "tzr": P["tz"]}
    from paper_2307_04528_gb300 import _lib as L_
    Hn = _handle(c, method=L_.MG_METHOD_STATIONARY)
    Hs = MGHandle(dev(P["tx"]), dev(P["ty"]), dev(P["tz"]), dev(P["h"]),
                  method=L_.MG_METHOD_STATIONARY)
    r = dev(np.random.default_rng(5).standard_normal(P["h"].shape))
    assert rel_inf(host(Hn.apply(r)), host(Hs.apply(r))) <= 1e-13
    assert rel_inf(host(Hn.apply(r, transpose=True)), host(Hs.apply(r))) <= 1e-13
    assert rel_inf(host(Hn.vcycle(r)), host(Hs.vcycle(r))) <= 1e-11
    xn, i1 = Hn.solve(dev(P["b"]), tol=1e-10)
    xs, i2 = Hs.solve(dev(P["b"]), tol=1e-10)
    assert rel_2(host(xn), host(xs)) <= 1e-9 and abs(i1["iterations"] - i2["iterations"]) <= 1


def test_coefficient_gradient_matches_the_oracle():
    P = _ns_problem(96, 46, 12)
    H = _handle(P)
    L, _, _ = _oracle(P)
    rng = np.random.default_rng(6)
    lam, x = rng.standard_normal(P["h"].shape), rng.standard_normal(P["h"].shape)
    got = H.coeff_grad(dev(lam), dev(x))
    for name, g, w in zip(NAMES, got, N.coeff_grad(L[0], lam, x)):
        assert rel_inf(host(g), w) <= 1e-15, name


@pytest.mark.parametrize("mixed", [False, True])
def test_differentiable_solve_against_dense_adjoint(mixed):
    """ns_solve_fn's gradients (forward solve, adjoint solve on H^T's
    hierarchy, the seven-array kernel; FP64 or with FP32 multigrid inside
    FP64 refinement) against the oracle's gradient formula at the dense
    solutions x = H^{-1} b and lam = H^{-T} g."""
    from paper_2307_04528_gb300.solver import ns_solve_fn
    P = _ns_problem(16, 8, 4, seed=23)
    L, _, _ = _oracle(P, levels=2)
    n = P["h"].size
    A = np.empty((n, n))
    e = np.zeros(n)
    for col in range(n):
        e[col] = 1.0
        A[:, col] = N.apply(L[0], e.reshape(P["h"].shape)).ravel()
        e[col] = 0.0
    g = np.random.default_rng(7).standard_normal(P["h"].shape)
    xs = np.linalg.solve(A, P["b"].ravel()).reshape(P["h"].shape)
    lam = np.linalg.solve(A.T, g.ravel()).reshape(P["h"].shape)
    want = dict(zip(NAMES, N.coeff_grad(L[0], lam, xs)))
    ts = {k: dev(P[k]).requires_grad_(True) for k in NAMES}
    b = dev(P["b"]).requires_grad_(True)
    x = ns_solve_fn(b, *(ts[k] for k in NAMES), tol=1e-11, floor_accept=1e-9, mixed=mixed,
                    levels=2)
    assert rel_2(host(x), xs) <= 1e-9
    (x * dev(g)).sum().backward()
    assert rel_2(host(b.grad), lam) <= 1e-8
    for k in NAMES:
        assert rel_2(host(ts[k].grad), want[k]) <= 1e-7, k


def test_bad_inputs_are_reported():
    from paper_2307_04528_gb300 import _lib as L_
    P = _ns_problem(32, 16, 4)
    for key, where, val in (("h", (0, 0, 0), -1.0), ("txr", (1, 2, 3), -0.5),
                            ("tyr", (0, 15, 2), 1.0), ("tzr", (3, 1, 1), 1.0),
                            ("tx", (1, 1, 1), np.nan)):
        Q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in P.items()}
        Q[key][where] = val
        with pytest.raises(L_.MGError) as ei:
            _handle(Q)
        assert ei.value.status == L_.MG_ERR_COEFF, key
    # a column sum that turns negative: a row couples more strongly back into
    # a cell than the cell's own mass allows
    Q = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in P.items()}
    Q["txr"][2, 5, 7] += 1e3 * Q["h"][2, 5, 7] + 1e3 * Q["tx"][2, 5, 7]
    with pytest.raises(L_.MGError) as ei:
        _handle(Q)
    assert ei.value.status == L_.MG_ERR_COEFF
    H = _handle(P)
    b = dev(P["b"])
    b[0, 0, 0] = float("nan")
    with pytest.raises(L_.MGError) as ei:
        H.solve(b)
    assert ei.value.status == L_.MG_ERR_NONFINITE
    x, info = H.solve(dev(P["b"]), tol=1e-10)  # still usable
    assert info["status"] == 0


def test_operational_size_properties():
    """1536 x 1152 x 70 (the operational-size workload with transport):
    <H x, y> = <x, H^T y> to rounding, and both H and H^T solve to 1e-10
    with BiCGStab preconditioned by the V-cycle."""
    P = _ns_problem(1536, 1152, 70, seed=24, sigma=0.2)
    H = _handle(P)
    del P["fx"], P["fy"], P["fz"]
    rng = torch.Generator(device="cuda").manual_seed(8)
    x = torch.randn(P["h"].shape, dtype=torch.float64, device="cuda", generator=rng)
    y = torch.randn(P["h"].shape, dtype=torch.float64, device="cuda", generator=rng)
    hx = H.apply(x)
    a = float(torch.dot(hx.ravel(), y.ravel()))
    b_ = float(torch.dot(x.ravel(), H.apply(y, transpose=True).ravel()))
    assert abs(a - b_) <= 1e-12 * float(torch.linalg.vector_norm(hx) * torch.linalg.vector_norm(y))
    del hx, x, y
    b = dev(P["b"])
    for tr in (False, True):
        xs, info = H.solve(b, tol=1e-10, transpose=tr)
        assert info["status"] == 0 and info["rel_res"] <= 1e-10, (tr, info)
        assert info["iterations"] <= 25, (tr, info)
        r = b - H.apply(xs, transpose=tr)
        assert float(torch.linalg.vector_norm(r) / torch.linalg.vector_norm(b)) <= 1.5e-10


# ----------------------------------------------------------------- mixed precision
def _ns_float(levels, scale):
    """The oracle's levels in FP32: every array scaled by the handle's power of
    two and rounded, as the library builds its FP32 hierarchy from FP64."""
    out = []
    for L in levels:
        arrs = [np.ascontiguousarray(a * scale, dtype=np.float32) for a in L.arrays()]
        out.append(N.NSLevel(*arrs, L.geo))
    return out


@pytest.mark.parametrize("shape", SHAPES)
def test_fp32_vcycles_of_h_and_its_transpose(shape):
    """The FP32 V-cycle of H and of H^T element by element against the oracle
    run in float32 on the same scaled levels (the symmetric FP32 cycle's
    tolerances: 1e-4 max-norm, 2e-5 2-norm), and against the FP64 cycle / c."""
    from paper_2307_04528_gb300 import _lib as L_
    P = _ns_problem(*shape)
    H = _handle(P, mixed=1)
    L, T, p = _oracle(P)
    c = H.fp32_scale
    _, ex = np.frexp(max(float(np.max(np.abs(a))) for lv in L + T for a in lv.arrays()))
    assert c == float(np.ldexp(1.0, -int(ex)))
    r = np.random.default_rng(40).standard_normal(P["h"].shape).astype(np.float32)
    for tr, levs in ((False, L), (True, T)):
        got = host(H.vcycle(dev(r, torch.float32), transpose=tr, prec=L_.MG_PREC_FP32))
        ref = N.vcycle(_ns_float(levs, c), r, p)
        assert ref.dtype == np.float32
        assert rel_inf(got, ref) <= 1e-4, tr
        assert rel_2(got, ref) <= 2e-5, tr
        e64 = host(H.vcycle(dev(r.astype(np.float64)), transpose=tr))
        assert rel_2(got * c, e64) <= 1e-4, tr


@pytest.mark.parametrize("method", ["stationary", "bicgstab"])
@pytest.mark.parametrize("transpose", [False, True])
def test_mixed_solves_reach_the_fp64_solution(method, transpose):
    """FP32 multigrid inside FP64 refinement reaches 1e-10 for H and H^T and
    the oracle's FP64 solution."""
    from paper_2307_04528_gb300 import _lib as L_
    P = _ns_problem(96, 46, 12)
    code = L_.MG_METHOD_STATIONARY if method == "stationary" else L_.MG_METHOD_BICGSTAB
    H = _handle(P, method=code, mixed=1)
    L, T, _ = _oracle(P)
    x, info = H.solve_mixed(dev(P["b"]), tol=1e-10, transpose=transpose)
    xo, _, st = N.solve(T if transpose else L, P["b"], 1e-11, O.MGParams(method=method))
    assert st == N.OK and info["status"] == 0
    assert info["rel_res"] <= 1e-10 and info["iterations"] <= 6
    assert rel_2(host(x), xo) <= 1e-8
    A = T[0] if transpose else L[0]
    true = np.linalg.norm(N.residual(A, P["b"], host(x))) / np.linalg.norm(P["b"])
    assert true <= 1.5e-10


def test_mixed_operational_size():
    """1536 x 1152 x 70 with transport: the mixed solves of H and H^T reach
    1e-10 in a few refinement steps, and their solutions agree with the FP64
    solves' to the tolerance's order."""
    P = _ns_problem(1536, 1152, 70, seed=24, sigma=0.2)
    H = _handle(P, mixed=1)
    del P["fx"], P["fy"], P["fz"]
    b = dev(P["b"])
    for tr in (False, True):
        xm, im = H.solve_mixed(b, tol=1e-10, transpose=tr)
        assert im["status"] == 0 and im["rel_res"] <= 1e-10 and im["iterations"] <= 6, (tr, im)
        x64, i64 = H.solve(b, tol=1e-10, transpose=tr)
        diff = float(torch.linalg.vector_norm(xm - x64) / torch.linalg.vector_norm(x64))
        assert diff <= 1e-7, (tr, diff)


@pytest.mark.parametrize("transpose", [False, True])
def test_fp32_sweeps_on_every_level(transpose):
    """Every level's FP32 sweeps (from zero and with a guess) of H and H^T
    against the oracle's float32 sweeps on the same scaled levels."""
    from paper_2307_04528_gb300 import _lib as L_
    P = _ns_problem(96, 46, 12)
    H = _handle(P, mixed=1)
    L, T, p = _oracle(P)
    levs = _ns_float(T if transpose else L, H.fp32_scale)
    rng = np.random.default_rng(41)
    for l, lev in enumerate(levs):
        b = rng.standard_normal(lev.shape).astype(np.float32)
        u = rng.standard_normal(lev.shape).astype(np.float32)
        f32 = lambda a: dev(a, torch.float32)
        z = H.level_smooth(l, f32(b), None, transpose=transpose, prec=L_.MG_PREC_FP32)
        assert rel_inf(host(z), N.smooth_from_zero(lev, b, p.omega)) <= 2e-5, (l, "zero")
        s = H.level_smooth(l, f32(b), f32(u), transpose=transpose, prec=L_.MG_PREC_FP32)
        assert rel_inf(host(s), N.smooth(lev, b, u, p.omega)) <= 2e-5, (l, "guess")


@pytest.mark.parametrize("shape,params", [((32, 16, 192), {}), ((48, 24, 33), {}),
                                          ((64, 32, 1), {}), ((16, 8, 5), {"levels": 1}),
                                          ((4, 2, 3), {})],
                         ids=["nz192", "nz33", "nz1", "one-level", "nlon4"])
def test_edge_shapes(shape, params):
    """The largest column (nz = 192), a layer count that is not a multiple
    of the warp width, a single layer (no vertical couplings), a single-level
    hierarchy (the coarse sweeps are the whole cycle) and the smallest grid:
    both hierarchies, the V-cycles and the BiCGStab solves of H and H^T
    against the oracle (nz = 192 and the 4 x 2 x 3 grid to 2e-8: their
    residual floors, the rounding of x times the vertical couplings, are
    ~6e-9 and ~3e-10)."""
    P = _ns_problem(*shape, seed=50 + shape[2])
    H = _handle(P, **params)
    L, T, p = _oracle(P, **params)
    assert H.num_levels == len(L)
    for l in range(len(L)):
        for tr, lev in ((False, L[l]), (True, T[l])):
            for name, g, w in zip(NAMES, H.level_coeffs(l, transpose=tr), lev.arrays()):
                assert rel_inf(host(g), w) <= 1e-15, (l, tr, name)
    r = np.random.default_rng(51).standard_normal(P["h"].shape)
    tol = 2e-8 if shape[2] == 192 or shape[0] == 4 else 1e-10
    for tr, levs in ((False, L), (True, T)):
        assert rel_inf(host(H.vcycle(dev(r), transpose=tr)), N.vcycle(levs, r, p)) <= 1e-11
        x, info = H.solve(dev(P["b"]), tol=tol, transpose=tr)
        xo, _, st = N.solve(levs, P["b"], tol / 10, O.MGParams(method="bicgstab", **params))
        assert info["status"] == 0 and st in (N.OK, N.NOT_CONVERGED)
        assert rel_2(host(x), xo) <= 100 * tol
