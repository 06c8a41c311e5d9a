"""GPU vs the CPU oracle at the operational grid 1536 x 1152 x 70 (sigma 0.2,
the benchmark's workload), through the handle the benchmark builds (default
parameters, FP32 hierarchy, CUDA graphs).

Every fine-level kernel of the V-cycle is compared element by element with
the oracle on the whole grid (FP64 1e-13, FP32 2e-5, integer structure and
coarse coefficients exact).  The oracle's V-cycle at this size is compared
to 1e-12.  Converged solutions are checked by the oracle's own FP64 residual
of the GPU solution, which must agree with the reported residual: a property
that holds at any size, where the oracle's full solve would take minutes.
"""
import numpy as np
import pytest
import torch

from gpu_common import dev, handle_for, host, oracle_levels, rel_2, rel_inf
from oracle import tpmg as O
from synthetic import make_problem

pytestmark = pytest.mark.gpu

SHAPE = (1536, 1152, 70)


@pytest.fixture(scope="module")
def full():
    P = make_problem(*SHAPE, 0.2, 3000)
    lev, p = oracle_levels(P)
    H = handle_for(P)
    return P, lev, p, H


def test_hierarchy_exact(full):
    P, lev, p, H = full
    assert H.num_levels == len(lev) == 9
    for l, ol in enumerate(lev):
        assert H.level_shape(l) == ol.shape
    for l in (0, 1, len(lev) - 1):
        for g, want in zip((host(t) for t in H.level_coeffs(l)), lev[l].coeffs()):
            assert np.array_equal(g, want)


def test_fine_level_kernels_fp64(full):
    P, lev, p, H = full
    f = lev[0]
    rng = np.random.default_rng(21)
    x = rng.standard_normal(f.shape)
    b = P["b"]
    assert rel_inf(host(H.level_apply(0, dev(x))), O.apply(f, x)) <= 1e-13
    assert rel_inf(host(H.level_residual(0, dev(b), dev(x))), O.residual(f, b, x)) <= 1e-13
    ref0 = np.zeros(f.shape)
    O.smooth(f, b, ref0, p.omega)
    assert rel_inf(host(H.level_smooth(0, dev(b))), ref0) <= 1e-13
    ref = x.copy()
    O.smooth(f, b, ref, p.omega)
    got, dot = H.level_smooth_dot(0, dev(b), dev(x))
    assert rel_inf(host(got), ref) <= 1e-13
    assert abs(dot - O.dot(b, ref)) <= 1e-12 * O.norm2(b) * O.norm2(ref)
    r = rng.standard_normal(f.shape)
    assert rel_inf(host(H.level_restrict(0, dev(r))), O.restrict(f, r)) <= 1e-13
    e = rng.standard_normal(lev[1].shape)
    ref = x.copy()
    O.prolong_add(f, e, ref)
    assert rel_inf(host(H.level_prolong_add(0, dev(e), dev(x))), ref) <= 1e-13


def test_fine_level_kernels_fp32(full):
    P, lev, p, H = full
    l32 = O.float_levels(lev)
    assert H.fp32_scale == l32[0].scale
    f = l32[0]
    rng = np.random.default_rng(22)
    x = rng.standard_normal(f.shape).astype(np.float32)
    b = rng.standard_normal(f.shape).astype(np.float32)
    f32 = lambda a: dev(a, torch.float32)
    assert rel_inf(host(H.level_apply(0, f32(x), prec=1)), O.apply(f, x)) <= 2e-5
    assert rel_inf(host(H.level_residual(0, f32(b), f32(x), prec=1)), O.residual(f, b, x)) <= 2e-5
    ref = x.copy()
    O.smooth(f, b, ref, np.float32(p.omega))
    assert rel_inf(host(H.level_smooth(0, f32(b), f32(x), prec=1)), ref) <= 2e-5
    got, dot = H.level_smooth_dot(0, f32(b), f32(x), prec=1)
    assert rel_inf(host(got), ref) <= 2e-5
    assert abs(dot - O.dot(b, ref)) <= 1e-5 * O.norm2(b) * O.norm2(ref)
    ref0 = np.zeros_like(x)
    O.smooth(f, b, ref0, np.float32(p.omega))
    assert rel_inf(host(H.level_smooth(0, f32(b), prec=1)), ref0) <= 2e-5
    assert rel_inf(host(H.level_restrict(0, f32(x), prec=1)), O.restrict(f, x)) <= 2e-5
    e = rng.standard_normal(l32[1].shape).astype(np.float32)
    ref = x.copy()
    O.prolong_add(f, e, ref)
    assert rel_inf(host(H.level_prolong_add(0, f32(e), f32(x), prec=1)), ref) <= 2e-5
    # the V-cycle's fused residual + restriction
    got = H.level_residual_restrict(0, f32(b), f32(x), prec=1)
    assert rel_inf(host(got), O.restrict(f, O.residual(f, b, x))) <= 2e-5
    two = H.level_restrict(0, H.level_residual(0, f32(b), f32(x), prec=1), prec=1)
    assert torch.equal(got, two)


def test_presmooth_restrict_fp32(full):
    """The V-cycle's residual + restriction after its sweep from zero (the
    form the benchmarked FP32 cycle runs) at full size: the band walk over
    1536-wide rows and every band of 8 coarse rows."""
    P, lev, p, H = full
    l32 = O.float_levels(lev)
    f = l32[0]
    b = np.random.default_rng(24).standard_normal(f.shape).astype(np.float32)
    u = H.level_smooth(0, dev(b, torch.float32), prec=1)
    got = host(H.level_presmooth_restrict(0, dev(b, torch.float32), u, prec=1))
    ref = O.restrict(f, O.presmooth_residual(f, b, host(u), np.float32(p.omega)))
    assert rel_inf(got, ref) <= 2e-5


def test_vcycle_fp32(full):
    """The whole FP32 V-cycle of the benchmarked mixed solve, element by
    element against the oracle's float V-cycle (bounds of the small-shape
    parity test)."""
    P, lev, p, H = full
    l32 = O.float_levels(lev)
    r = np.random.default_rng(25).standard_normal(lev[0].shape).astype(np.float32)
    got = host(H.vcycle(dev(r, torch.float32), prec=1))
    ref = O.vcycle(l32, r, p)
    assert rel_inf(got, ref) <= 1e-4
    assert rel_2(got, ref) <= 2e-5


def test_vcycle_fp64(full):
    P, lev, p, H = full
    r = np.random.default_rng(23).standard_normal(lev[0].shape)
    assert rel_inf(host(H.vcycle(dev(r))), O.vcycle(lev, r, p)) <= 1e-12


@pytest.mark.parametrize("mixed", [True, False], ids=["mixed", "fp64"])
def test_solution_residual_checked_by_oracle(full, mixed):
    """The benchmark's solve to 1e-10; the oracle's FP64 residual of the GPU
    solution agrees with the reported one and meets the tolerance."""
    P, lev, p, H = full
    b = dev(P["b"])
    x, info = (H.solve_mixed if mixed else H.solve)(b, tol=1e-10)
    assert info["status"] == 0 and info["rel_res"] <= 1e-10
    xr = host(x)
    rel = O.norm2(O.residual(lev[0], P["b"], xr)) / O.norm2(P["b"])
    assert rel <= 1e-10
    assert abs(rel - info["rel_res"]) <= 1e-12
