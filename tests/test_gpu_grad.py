"""Differentiable solve on the GPU: MGSolveFn (adjoint solve with the same
hierarchy + the fused coefficient-gradient kernel) against a dense-LU
reference gradient on 8x4x4 and central finite differences on 256x128x32
(step 1e-6 on unit directions; loss 0.5 ||W x||^2, W ~ U[0,1] seeded)."""
import numpy as np
import pytest
import torch

from gpu_common import dev, host, problem, rel_2, rel_inf
from oracle import tpmg as O
from test_oracle_pins import _dense_solve

pytestmark = pytest.mark.gpu


def _grads(P, W, tol=1e-12, mixed=False):
    from paper_2307_04528_gb300.solver import mg_solve_fn
    b, h, tx, ty, tz = (dev(P[k]).requires_grad_(True) for k in ("b", "h", "tx", "ty", "tz"))
    # the adjoint's smooth right-hand side floors near 6e-11: accepted below 1e-8
    x = mg_solve_fn(b, h, tx, ty, tz, tol=tol, floor_accept=1e-8, mixed=mixed)
    loss = 0.5 * torch.sum((dev(W) * x) ** 2)
    loss.backward()
    return x, {k: host(t.grad) for k, t in zip(("b", "h", "tx", "ty", "tz"), (b, h, tx, ty, tz))}


@pytest.mark.parametrize("mixed", [False, True])
def test_gradient_matches_dense_lu_8x4x4(mixed):
    """FP64 solves, or both solves with FP32 multigrid inside FP64
    refinement (mixed): the same gradient to the same bounds."""
    P = problem(8, 4, 4, sigma=0.1, seed=21)
    W = np.random.default_rng(22).uniform(0, 1, P["h"].shape)
    # the residual floor of this tiny grid is ~1e-11 (rounding of x times the
    # vertical couplings); the solution itself is far more accurate
    x, g = _grads(P, W, tol=5e-11, mixed=mixed)
    xd, _ = _dense_solve(P, P["b"])
    lam, _ = _dense_solve(P, W * W * xd)
    assert rel_2(host(x), xd) <= 1e-10
    assert rel_2(g["b"], lam) <= 1e-10
    assert rel_2(g["h"], -lam * xd) <= 1e-10
    lev = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], O.MGParams())
    gh, gtx, gty, gtz = O.coeff_grad(lev[0], lam, xd)
    for key, ref in (("tx", gtx), ("ty", gty)):
        assert rel_2(g[key], ref) <= 1e-9, key
    # vertical face gradients difference nearly equal values of x and lambda
    assert rel_2(g["tz"], gtz) <= 1e-6


def test_coeff_grad_kernel_parity():
    from paper_2307_04528_gb300.solver import MGHandle
    P = problem(96, 46, 9, sigma=0.2, seed=5)
    rng = np.random.default_rng(6)
    lam = rng.standard_normal(P["h"].shape)
    x = rng.standard_normal(P["h"].shape)
    H = MGHandle(dev(P["tx"]), dev(P["ty"]), dev(P["tz"]), dev(P["h"]))
    got = [host(t) for t in H.coeff_grad(dev(lam), dev(x))]
    lev = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], O.MGParams())
    ref = O.coeff_grad(lev[0], lam, x)
    for a, r in zip(got, ref):
        assert np.array_equal(a, r)


def test_gradient_central_differences_256x128x32():
    """64 unit directions each for b and h, step 1e-6, relative 1e-6."""
    from paper_2307_04528_gb300.solver import MGHandle
    P = problem(256, 128, 32, sigma=0.1, seed=4000)
    rng = np.random.default_rng(4001)
    W = dev(rng.uniform(0, 1, P["h"].shape))
    _, g = _grads(P, host(W), tol=1e-11)
    gb, gh = dev(g["b"]), dev(g["h"])
    b0 = dev(P["b"])
    coeffs = [dev(P[k]) for k in ("tx", "ty", "tz", "h")]
    H0 = MGHandle(*coeffs, maxit=40)  # 40 CG iterations: past the FP64 floor

    def loss_b(b):
        x, _ = H0.solve(b, tol=0.0, raise_on_error=False)
        return 0.5 * float(torch.sum((W * x) ** 2))

    def loss_h(h):
        H = MGHandle(coeffs[0], coeffs[1], coeffs[2], h, maxit=40)
        x, _ = H.solve(b0, tol=0.0, raise_on_error=False)
        return 0.5 * float(torch.sum((W * x) ** 2))

    eps = 1e-6
    gen = torch.Generator(device="cuda").manual_seed(7)
    nb = float(torch.linalg.vector_norm(gb))
    nh = float(torch.linalg.vector_norm(gh * coeffs[3]))
    worst_b = worst_h = 0.0
    for _ in range(64):
        d = torch.randn(b0.shape, generator=gen, device="cuda", dtype=torch.float64)
        d /= torch.linalg.vector_norm(d)
        fd = (loss_b(b0 + eps * d) - loss_b(b0 - eps * d)) / (2 * eps)
        worst_b = max(worst_b, abs(fd - float(torch.sum(gb * d))) / nb)
        fdh = (loss_h(coeffs[3] * (1 + eps * d)) - loss_h(coeffs[3] * (1 - eps * d))) / (2 * eps)
        worst_h = max(worst_h, abs(fdh - float(torch.sum(gh * coeffs[3] * d))) / nh)
    assert worst_b <= 1e-6, worst_b
    assert worst_h <= 1e-6, worst_h


def test_unconverged_solve_is_refused_unless_accepted():
    """A tolerance below the FP64 floor: refused by default, used with a
    warning when the caller opts in with floor_accept."""
    import warnings

    from paper_2307_04528_gb300 import _lib as L
    from paper_2307_04528_gb300.solver import MGFloorWarning, mg_solve_fn
    P = problem(32, 16, 8, sigma=0.1, seed=23)
    args = [dev(P[k]).requires_grad_(True) for k in ("b", "h", "tx", "ty", "tz")]
    with pytest.raises(L.MGError):
        mg_solve_fn(*args, tol=1e-18, maxit=30)
    with warnings.catch_warnings(record=True) as caught:
        warnings.simplefilter("always")
        x = mg_solve_fn(*args, tol=1e-18, floor_accept=1e-8, maxit=30)
        torch.sum(x * x).backward()
    assert sum(isinstance(w.message, MGFloorWarning) for w in caught) == 2
    assert args[0].grad is not None
