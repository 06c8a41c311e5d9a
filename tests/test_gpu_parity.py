"""GPU (libtpmg through its C ABI) vs the CPU oracle, element by element.

Tolerances: FP64 operator apply, residual, smoother sweep and transfers 1e-13
relative (max norm); a V-cycle 1e-12 (a composition of ~20 such steps);
converged FP64 and mixed-precision solutions 1e-10 relative 2-norm error.
FP32 kernels against the oracle's float instance: 2e-5 relative (rounding
order in single precision).  Integer structure (row maps, level shapes) and
the coarse coefficients (same summation order on both sides) are exact.
"""
import numpy as np
import pytest
import torch

from gpu_common import dev, handle_for, host, oracle_levels, problem, rel_2, rel_inf
from oracle import tpmg as O

pytestmark = pytest.mark.gpu

# several column tiles of 128 threads and a ragged tail; odd level counts
SHAPES = [(64, 32, 16), (96, 46, 9), (24, 10, 5), (256, 128, 12)]


@pytest.fixture(scope="module", params=SHAPES, ids=lambda s: "x".join(map(str, s)))
def case(request):
    P = problem(*request.param, sigma=0.2, seed=sum(request.param))
    lev, p = oracle_levels(P)
    H = handle_for(P)
    return P, lev, p, H


def test_hierarchy_shapes_and_coarse_coefficients_exact(case):
    P, lev, p, H = case
    assert H.num_levels == len(lev)
    for l, ol in enumerate(lev):
        assert H.level_shape(l) == ol.shape
        got = [host(t) for t in H.level_coeffs(l)]
        for g, want in zip(got, ol.coeffs()):
            assert np.array_equal(g, want)


def test_apply_and_residual_fp64(case):
    P, lev, p, H = case
    rng = np.random.default_rng(1)
    for l, ol in enumerate(lev):
        x = rng.standard_normal(ol.shape)
        b = rng.standard_normal(ol.shape)
        y = host(H.level_apply(l, dev(x)))
        assert rel_inf(y, O.apply(ol, x)) <= 1e-13
        r = host(H.level_residual(l, dev(b), dev(x)))
        assert rel_inf(r, O.residual(ol, b, x)) <= 1e-13
    y0 = host(H.apply(dev(lev[0].h * 0 + 1.0)))
    assert np.array_equal(y0, P["h"])  # H 1 = h exactly


def test_smoother_fp64(case):
    P, lev, p, H = case
    rng = np.random.default_rng(2)
    for l, ol in enumerate(lev):
        b = rng.standard_normal(ol.shape)
        u = rng.standard_normal(ol.shape)
        got0 = host(H.level_smooth(l, dev(b)))
        ref0 = np.zeros(ol.shape)
        O.smooth(ol, b, ref0, p.omega)
        assert rel_inf(got0, ref0) <= 1e-13
        got = host(H.level_smooth(l, dev(b), dev(u)))
        ref = u.copy()
        O.smooth(ol, b, ref, p.omega)
        assert rel_inf(got, ref) <= 1e-13


def test_smoother_with_fused_dot(case):
    """The V-cycle's last sweep with <b, u_out> fused: same sweep, and the
    inner product of the oracle's sweep result (FP64 1e-13, FP32 2e-5)."""
    P, lev, p, H = case
    rng = np.random.default_rng(12)
    for l, ol in enumerate(lev[:2]):
        b = rng.standard_normal(ol.shape)
        u = rng.standard_normal(ol.shape)
        got, dot = H.level_smooth_dot(l, dev(b), dev(u))
        ref = u.copy()
        O.smooth(ol, b, ref, p.omega)
        assert rel_inf(host(got), ref) <= 1e-13
        want = O.dot(b, ref)
        assert abs(dot - want) <= 1e-12 * O.norm2(b) * O.norm2(ref)
    l32 = O.float_levels(lev)
    b = rng.standard_normal(lev[0].shape).astype(np.float32)
    u = rng.standard_normal(lev[0].shape).astype(np.float32)
    got, dot = H.level_smooth_dot(0, dev(b, torch.float32), dev(u, torch.float32), prec=1)
    ref = u.copy()
    O.smooth(l32[0], b, ref, np.float32(p.omega))
    assert rel_inf(host(got), ref) <= 2e-5
    assert abs(dot - O.dot(b, ref)) <= 1e-5 * O.norm2(b) * O.norm2(ref)


def _sweeps_from_zero(ol, b, sweeps, omega):
    ref = np.zeros_like(b)
    for _ in range(sweeps):
        O.smooth(ol, b, ref, omega)
    return ref


def test_relax_and_coarsest_solve(case):
    """`coarse_iters` sweeps from zero on the coarsest level (the V-cycle's
    coarsest-level solve: one launch, the level in shared memory in FP32) and
    on the finest (one launch per sweep), FP64 1e-12 and FP32 2e-5 against
    the oracle's sweeps repeated (FP32 rounding drift over 12 sweeps measured
    at ~1e-6 on these shapes)."""
    P, lev, p, H = case
    l32 = O.float_levels(lev)
    rng = np.random.default_rng(13)
    for l in sorted({0, len(lev) - 1}):
        b = rng.standard_normal(lev[l].shape)
        got = host(H.level_relax(l, dev(b), p.coarse_iters))
        assert rel_inf(got, _sweeps_from_zero(lev[l], b, p.coarse_iters, p.omega)) <= 1e-12
        b32 = b.astype(np.float32)
        got = host(H.level_relax(l, dev(b32, torch.float32), p.coarse_iters, prec=1))
        want = _sweeps_from_zero(l32[l], b32, p.coarse_iters, np.float32(p.omega))
        assert rel_inf(got, want) <= 2e-5
    b = rng.standard_normal(lev[-1].shape)
    one = host(H.level_relax(len(lev) - 1, dev(b), 1))
    assert rel_inf(one, _sweeps_from_zero(lev[-1], b, 1, p.omega)) <= 1e-13
    b32 = b.astype(np.float32)
    for sweeps in (1, 3):
        got = host(H.level_relax(len(lev) - 1, dev(b32, torch.float32), sweeps, prec=1))
        want = _sweeps_from_zero(l32[-1], b32, sweeps, np.float32(p.omega))
        assert rel_inf(got, want) <= 2e-5


@pytest.mark.parametrize("shape,levels", [((64, 32, 16), 3), ((96, 46, 9), 2), ((64, 32, 16), 0)])
def test_coarse_pcg(shape, levels):
    """coarse_method = PCG: the coarsest-level solve against the oracle's
    coarse_pcg (FP64 1e-10; FP32 2e-5, its FP32 rounding drift measured at
    ~5e-7 on these levels), the FP64 V-cycle against the oracle's (1e-10),
    and a 3-level FP64 and mixed solve to 1e-10 against the oracle's FP64
    solution (1e-9)."""
    P = problem(*shape, sigma=0.2, seed=sum(shape) + levels)
    lev, p = oracle_levels(P, levels=levels, coarse_method="pcg")
    H = handle_for(P, levels=levels, coarse_method=1)
    assert H.num_levels == len(lev)
    l32 = O.float_levels(lev)
    rng = np.random.default_rng(16)
    b = rng.standard_normal(lev[-1].shape)
    got = host(H.coarse_solve(dev(b)))
    assert rel_inf(got, O.coarse_pcg(lev[-1], b, p.coarse_iters)) <= 1e-10
    b32 = b.astype(np.float32)
    got = host(H.coarse_solve(dev(b32, torch.float32), prec=1))
    assert rel_inf(got, O.coarse_pcg(l32[-1], b32, p.coarse_iters)) <= 2e-5
    r = rng.standard_normal(lev[0].shape)
    assert rel_inf(host(H.vcycle(dev(r))), O.vcycle(lev, r, p)) <= 1e-10
    if levels == 3:
        xr, _, sr = O.solve(lev, P["b"], 1e-11, params=p)
        assert sr == O.OK
        for fn in (H.solve, H.solve_mixed):
            x, info = fn(dev(P["b"]), tol=1e-10)
            assert info["status"] == 0 and info["rel_res"] <= 1e-10
            assert rel_2(host(x), xr) <= 1e-9


@pytest.mark.parametrize("shape,levels", [((64, 32, 16), 3), ((96, 46, 9), 2), ((64, 32, 16), 0)])
def test_coarse_chebyshev(shape, levels):
    """coarse_method = Chebyshev: the coarsest-level solve against the
    oracle's coarse_chebyshev (a fixed polynomial: FP64 1e-11, FP32 2e-5),
    the FP64 V-cycle against the oracle's (1e-10), and a 3-level FP64 and
    mixed solve to 1e-10 against the oracle's FP64 solution (1e-9)."""
    P = problem(*shape, sigma=0.2, seed=sum(shape) + 2 * levels)
    lev, p = oracle_levels(P, levels=levels, coarse_method="chebyshev")
    H = handle_for(P, levels=levels, coarse_method=2)
    assert H.num_levels == len(lev)
    l32 = O.float_levels(lev)
    rng = np.random.default_rng(17)
    b = rng.standard_normal(lev[-1].shape)
    got = host(H.coarse_solve(dev(b)))
    assert rel_inf(got, O.coarse_chebyshev(lev[-1], b, p.coarse_iters)) <= 1e-11
    b32 = b.astype(np.float32)
    got = host(H.coarse_solve(dev(b32, torch.float32), prec=1))
    assert rel_inf(got, O.coarse_chebyshev(l32[-1], b32, p.coarse_iters)) <= 2e-5
    r = rng.standard_normal(lev[0].shape)
    assert rel_inf(host(H.vcycle(dev(r))), O.vcycle(lev, r, p)) <= 1e-10
    if levels == 3:
        xr, _, sr = O.solve(lev, P["b"], 1e-11, params=p)
        assert sr == O.OK
        for fn in (H.solve, H.solve_mixed):
            x, info = fn(dev(P["b"]), tol=1e-10)
            assert info["status"] == 0 and info["rel_res"] <= 1e-10
            assert rel_2(host(x), xr) <= 1e-9


def test_isotropy_stopping_rule():
    """levels = -1 (coarsen until the couplings are within iso_ratio): the
    same depth and shapes as the oracle's rule, on a system with a large
    Helmholtz term (stops early) and on the lat-lon workload (full depth),
    and the solve against the oracle's solution."""
    for hscale, shape in ((1e4, (64, 32, 16)), (1.0, (96, 46, 9))):
        P = problem(*shape, sigma=0.2, seed=61)
        P = dict(P, h=P["h"] * hscale)
        lev, p = oracle_levels(P, levels=-1)
        H = handle_for(P, levels=-1)
        assert H.num_levels == len(lev)
        for l, ol in enumerate(lev):
            assert H.level_shape(l) == ol.shape
        xr, _, sr = O.solve(lev, P["b"], 1e-11, params=p)
        assert sr == O.OK
        x, info = H.solve_mixed(dev(P["b"]), tol=1e-10)
        assert info["status"] == 0 and rel_2(host(x), xr) <= 1e-9


def test_coarsest_solve_beyond_shared_memory():
    """A shallow hierarchy whose coarsest level (40 x 30 x 32 cells) exceeds
    one block's shared memory: the FP32 coarsest-level solve runs from
    global memory (one block, 32 warps); odd sweep counts end in out."""
    P = problem(128, 64, 40, sigma=0.2, seed=232)
    lev, p = oracle_levels(P, levels=3)
    H = handle_for(P, levels=3)
    assert H.num_levels == 3 and H.level_shape(2) == (40, 30, 32)
    l32 = O.float_levels(lev)
    rng = np.random.default_rng(14)
    b32 = rng.standard_normal(lev[2].shape).astype(np.float32)
    for sweeps in (p.coarse_iters, 3):
        got = host(H.level_relax(2, dev(b32, torch.float32), sweeps, prec=1))
        want = _sweeps_from_zero(l32[2], b32, sweeps, np.float32(p.omega))
        assert rel_inf(got, want) <= 2e-5


def test_residual_restrict_fused(case):
    """R (b - H u) in one pass on every level: against the oracle's residual
    then restriction (FP64 1e-13, FP32 2e-5), and equal to the library's own
    two passes exactly (the same operations in the same order).  A buffer
    one value off alignment takes the two-pass path."""
    P, lev, p, H = case
    l32 = O.float_levels(lev)
    rng = np.random.default_rng(15)
    for l in range(len(lev) - 1):
        b = rng.standard_normal(lev[l].shape)
        u = rng.standard_normal(lev[l].shape)
        got = host(H.level_residual_restrict(l, dev(b), dev(u)))
        assert rel_inf(got, O.restrict(lev[l], O.residual(lev[l], b, u))) <= 1e-13
        b32, u32 = dev(b, torch.float32), dev(u, torch.float32)
        got = H.level_residual_restrict(l, b32, u32, prec=1)
        want = O.restrict(l32[l], O.residual(l32[l], host(b32), host(u32)))
        assert rel_inf(host(got), want) <= 2e-5
        two = H.level_restrict(l, H.level_residual(l, b32, u32, prec=1), prec=1)
        assert torch.equal(got, two)
    buf = torch.empty(lev[0].size + 1, dtype=torch.float32, device="cuda")
    b_odd = buf[1:].view(lev[0].shape)
    b_odd.copy_(dev(rng.standard_normal(lev[0].shape), torch.float32))
    u32 = dev(rng.standard_normal(lev[0].shape), torch.float32)
    got = H.level_residual_restrict(0, b_odd, u32, prec=1)
    assert torch.equal(got, H.level_restrict(0, H.level_residual(0, b_odd, u32, prec=1), prec=1))


def test_presmooth_restrict(case):
    """The V-cycle's restricted residual after its sweep from zero, u = omega
    H_z^{-1} b, taken as (1 - omega) b plus u's horizontal couplings: against
    the oracle's presmooth_residual then restriction on every level (FP64
    1e-13, FP32 2e-5); unaligned buffers give the aligned result exactly."""
    P, lev, p, H = case
    l32 = O.float_levels(lev)
    rng = np.random.default_rng(17)
    for l in range(len(lev) - 1):
        b = rng.standard_normal(lev[l].shape)
        u = np.zeros_like(b)
        O.smooth(lev[l], b, u, p.omega)
        got = host(H.level_presmooth_restrict(l, dev(b), dev(u)))
        want = O.restrict(lev[l], O.presmooth_residual(lev[l], b, u, p.omega))
        assert rel_inf(got, want) <= 1e-13
        b32 = b.astype(np.float32)
        u32 = np.zeros_like(b32)
        O.smooth(l32[l], b32, u32, np.float32(p.omega))
        got = H.level_presmooth_restrict(l, dev(b32, torch.float32), dev(u32, torch.float32),
                                         prec=1)
        want = O.restrict(l32[l], O.presmooth_residual(l32[l], b32, u32, np.float32(p.omega)))
        assert rel_inf(host(got), want) <= 2e-5
    n = lev[0].size
    buf = torch.empty(2 * n + 1, dtype=torch.float32, device="cuda")
    b_odd, u_odd = buf[1:n + 1].view(lev[0].shape), buf[n + 1:].view(lev[0].shape)
    b_odd.copy_(dev(rng.standard_normal(lev[0].shape), torch.float32))
    u_odd.copy_(dev(rng.standard_normal(lev[0].shape), torch.float32))
    got = H.level_presmooth_restrict(0, b_odd, u_odd, prec=1)
    assert torch.equal(got, H.level_presmooth_restrict(0, b_odd.clone(), u_odd.clone(), prec=1))


def test_vcycle_unaligned_input(case):
    """mg_vcycle on a right-hand side one value off alignment (copied into
    the level's work vector for the fused pass) gives the aligned result."""
    P, lev, p, H = case
    r = np.random.default_rng(18).standard_normal(lev[0].shape)
    buf = torch.empty(lev[0].size + 1, dtype=torch.float64, device="cuda")
    r_odd = buf[1:].view(lev[0].shape)
    r_odd.copy_(dev(r))
    assert torch.equal(H.vcycle(r_odd), H.vcycle(dev(r)))


def test_transfers_fp64(case):
    P, lev, p, H = case
    rng = np.random.default_rng(3)
    for l in range(len(lev) - 1):
        f, c = lev[l], lev[l + 1]
        r = rng.standard_normal(f.shape)
        assert rel_inf(host(H.level_restrict(l, dev(r))), O.restrict(f, r)) <= 1e-13
        e = rng.standard_normal(c.shape)
        u = rng.standard_normal(f.shape)
        ref = u.copy()
        O.prolong_add(f, e, ref)
        assert rel_inf(host(H.level_prolong_add(l, dev(e), dev(u))), ref) <= 1e-13


def test_fp32_kernels(case):
    P, lev, p, H = case
    l32 = O.float_levels(lev)
    assert H.fp32_scale == l32[0].scale
    rng = np.random.default_rng(4)
    f32 = lambda a: dev(a, torch.float32)
    for l, ol in enumerate(l32):
        x = rng.standard_normal(ol.shape).astype(np.float32)
        b = rng.standard_normal(ol.shape).astype(np.float32)
        assert rel_inf(host(H.level_apply(l, f32(x), prec=1)), O.apply(ol, x)) <= 2e-5
        ref = x.copy()
        O.smooth(ol, b, ref, np.float32(p.omega))
        assert rel_inf(host(H.level_smooth(l, f32(b), f32(x), prec=1)), ref) <= 2e-5
        ref0 = np.zeros_like(x)
        O.smooth(ol, b, ref0, np.float32(p.omega))
        assert rel_inf(host(H.level_smooth(l, f32(b), prec=1)), ref0) <= 2e-5
        if l + 1 < len(l32):
            assert rel_inf(host(H.level_restrict(l, f32(x), prec=1)), O.restrict(ol, x)) <= 2e-5


def test_dir_apply_every_level(case):
    """The CG step d_new = z + beta d_old, q = H d_new, <d_new, q> (the
    register-pipeline kernel at these sizes) against the oracle's apply."""
    P, lev, p, H = case
    rng = np.random.default_rng(9)
    for l, ol in enumerate(lev):
        z = rng.standard_normal(ol.shape)
        d = rng.standard_normal(ol.shape)
        dn, q, dot = H.level_dir_apply(l, dev(z), dev(d), 0.37)
        dref = host(dn)
        assert rel_inf(dref, z + 0.37 * d) <= 1e-15
        assert rel_inf(host(q), O.apply(ol, dref)) <= 1e-13
        assert abs(dot - O.dot(dref, host(q))) <= 1e-12 * O.norm2(dref) * O.norm2(host(q))
        dn, q, _ = H.level_dir_apply(l, dev(z), None)
        assert np.array_equal(host(dn), z) and rel_inf(host(q), O.apply(ol, z)) <= 1e-13


# FP32 V-cycle against the oracle's float V-cycle: both run V(1,1) with the
# same steps in FP32 but different rounding orders (fused multiply-adds, the
# warp-scan column sweeps of the small levels); each step is good to ~1e-6
# relative and the cycle composes ~2 L + 12 of them with a contraction, so
# 1e-4 in the max norm and 2e-5 in the 2-norm leave a margin of ~10.
FP32_VCYCLE_INF, FP32_VCYCLE_2 = 1e-4, 2e-5


def test_vcycle_fp32(case):
    P, lev, p, H = case
    l32 = O.float_levels(lev)
    r = np.random.default_rng(31).standard_normal(lev[0].shape).astype(np.float32)
    got = host(H.vcycle(dev(r, torch.float32), prec=1))
    ref = O.vcycle(l32, r, p)
    assert rel_inf(got, ref) <= FP32_VCYCLE_INF
    assert rel_2(got, ref) <= FP32_VCYCLE_2
    # the FP32 hierarchy holds c H: its cycle approximates the FP64 one / c
    e64 = host(H.vcycle(dev(r.astype(np.float64))))
    assert rel_2(got * l32[0].scale, e64) <= 1e-4


def test_vcycle_fp64(case):
    P, lev, p, H = case
    rng = np.random.default_rng(5)
    r = rng.standard_normal(lev[0].shape)
    assert rel_inf(host(H.vcycle(dev(r))), O.vcycle(lev, r, p)) <= 1e-12


@pytest.mark.parametrize("method", ["cg", "stationary"])
def test_solve_fp64_matches_oracle(method):
    P = problem(64, 32, 16, sigma=0.1, seed=1000)
    lev, p = oracle_levels(P, method=method)
    H = handle_for(P, method=0 if method == "cg" else 1)
    xr, hr, sr = O.solve(lev, P["b"], 1e-11, params=p)
    x, info = H.solve(dev(P["b"]), tol=1e-11)
    assert sr == O.OK and info["status"] == 0
    assert info["rel_res"] <= 1e-11
    assert abs(len(info["history"]) - len(hr)) <= 1
    assert rel_2(host(x), xr) <= 1e-10
    # the residual the library reports is the oracle's residual of its x
    assert O.norm2(O.residual(lev[0], P["b"], host(x))) / O.norm2(P["b"]) <= 1.5e-11


def test_solve_mixed_matches_fp64_oracle():
    P = problem(64, 32, 16, sigma=0.1, seed=1000)
    lev, p = oracle_levels(P)
    H = handle_for(P)
    xr, _, _ = O.solve(lev, P["b"], 1e-12, params=p)
    x, info = H.solve_mixed(dev(P["b"]), tol=1e-11)
    assert info["status"] == 0 and info["rel_res"] <= 1e-11
    assert rel_2(host(x), xr) <= 1e-10
    xo, ho, so = O.solve_mixed(lev, P["b"], 1e-11, params=p)
    assert so == O.OK
    assert abs(len(info["history"]) - len(ho)) <= 2


def test_degenerate_single_layer_and_two_rows():
    for shape in [(16, 2, 3), (32, 8, 1)]:
        P = problem(*shape, sigma=0.1, seed=3)
        lev, p = oracle_levels(P)
        H = handle_for(P)
        x, info = H.solve(dev(P["b"]), tol=1e-10)
        xr, _, _ = O.solve(lev, P["b"], 1e-10, params=p)
        assert info["status"] == 0
        assert rel_2(host(x), xr) <= 1e-9


def test_zero_rhs_gives_zero():
    P = problem(16, 8, 4)
    H = handle_for(P)
    x, info = H.solve(torch.zeros(P["h"].shape, dtype=torch.float64, device="cuda"))
    assert info["status"] == 0 and float(x.abs().max()) == 0.0
