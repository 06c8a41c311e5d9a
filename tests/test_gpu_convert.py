"""The precision changes of the mixed-precision refinement (mg_cast_fp32,
mg_update_fp64): with a power-of-two scale they run in integer arithmetic,
and must give the IEEE 754 results bit for bit.  The reference is numpy on
the host (round to nearest, ties to even, gradual underflow, overflow to
infinity), over values chosen to hit every branch: random magnitudes across
the binary64 range, exact halfway cases and their neighbours, the overflow
threshold, the subnormal range and its lower edge, zeros, infinities and a
NaN; the 16-byte vector kernels (length a multiple of 4) and the scalar
ones (odd length, misaligned view) alike."""
import math

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

SCALES = [1.0, 2.0 ** -7, 2.0 ** 13, 2.0 ** -100, 2.0 ** 60, 3.0]  # 3: the FP64 product path


def _special_values(rng):
    v = list(rng.standard_normal(6000) * np.exp2(rng.integers(-170, 150, 6000)))
    for _ in range(800):  # halfway between neighbouring binary32 values, and either side
        f = np.float32(rng.standard_normal() * 2.0 ** int(rng.integers(-149, 127)))
        if not np.isfinite(f) or f == 0:
            continue
        nxt = float(np.nextafter(f, np.float32(np.inf) if f > 0 else np.float32(-np.inf)))
        if not math.isfinite(nxt):
            continue
        mid = (float(f) + nxt) / 2
        v += [mid, math.nextafter(mid, 0.0), math.nextafter(mid, math.inf),
              math.nextafter(mid, -math.inf)]
    fmax = float(np.finfo(np.float32).max)
    v += [fmax, fmax * (1 + 2.0 ** -25), fmax * (1 + 2.0 ** -24),
          math.nextafter(fmax * (1 + 2.0 ** -24), 0.0), 2.0 ** 128, -2.0 ** 128,
          2.0 ** -149, 2.0 ** -150, math.nextafter(2.0 ** -150, 1.0), 2.0 ** -151,
          3 * 2.0 ** -151, 2.0 ** -126, math.nextafter(2.0 ** -126, 0.0), 5e-324, -5e-324,
          0.0, -0.0, math.inf, -math.inf, 1e300, -1e-300]
    return np.array(v, dtype=np.float64)


def _bits32(a):
    return np.asarray(a, dtype=np.float32).view(np.uint32)


def _bits64(a):
    return np.asarray(a, dtype=np.float64).view(np.uint64)


@pytest.mark.parametrize("scale", SCALES)
def test_cast_fp32_rounds_as_ieee(scale):
    from paper_2307_04528_gb300.solver import cast_fp32
    x = _special_values(np.random.default_rng(11))
    x = np.concatenate([x, [np.nan]])
    x = x[: len(x) // 4 * 4]
    with np.errstate(over="ignore", under="ignore"):
        ref = (x * scale).astype(np.float32)
    for n in (len(x), len(x) - 1):  # vector kernel, scalar kernel
        got = cast_fp32(torch.from_numpy(x[:n]).cuda(), scale).cpu().numpy()
        fin = ~np.isnan(ref[:n])
        assert np.array_equal(_bits32(got[fin]), _bits32(ref[:n][fin]))
        assert np.isnan(got[~fin]).all()
    # a view starting 8 bytes into its buffer (not 16-byte aligned)
    buf = torch.from_numpy(np.concatenate([[0.0], x])).cuda()
    got = cast_fp32(buf[1:], scale).cpu().numpy()
    fin = ~np.isnan(ref)
    assert np.array_equal(_bits32(got[fin]), _bits32(ref[fin]))


@pytest.mark.parametrize("scale", [1.0, 2.0 ** -20, 2.0 ** 30, 0.75])
def test_update_fp64_is_one_rounding(scale):
    from paper_2307_04528_gb300.solver import update_fp64
    rng = np.random.default_rng(12)
    n = 8192
    x = rng.standard_normal(n) * np.exp2(rng.integers(-60, 60, n))
    e = (rng.standard_normal(n) * np.exp2(rng.integers(-140, 120, n))).astype(np.float32)
    e[:8] = [0.0, -0.0, 1e-45, -1e-45, 1.1754942e-38, 3.4028235e38, 7e-40, -3e-42]
    ref = x + scale * e.astype(np.float64)  # exact product, one rounding
    for m in (n, n - 3):
        xt = torch.from_numpy(x[:m].copy()).cuda()
        got = update_fp64(xt, torch.from_numpy(e[:m]).cuda(), scale).cpu().numpy()
        assert np.array_equal(_bits64(got), _bits64(ref[:m]))


def test_update_fp64_widens_special_values():
    """x = 0 exposes the widened value itself: signed zeros, binary32
    subnormals (renormalised in binary64) and infinities."""
    from paper_2307_04528_gb300.solver import update_fp64
    e = np.array([0.0, -0.0, 1e-45, -1e-45, 2.0 ** -130, 1.1754942e-38, 3.4028235e38, np.inf,
                  -np.inf, 1.5], dtype=np.float32)
    x = torch.zeros(len(e), dtype=torch.float64, device="cuda")
    got = update_fp64(x, torch.from_numpy(e).cuda(), 1.0).cpu().numpy()
    assert np.array_equal(got, e.astype(np.float64))
    assert np.array_equal(np.signbit(got[2:]), np.signbit(e[2:].astype(np.float64)))


def test_conversion_arguments_checked():
    from paper_2307_04528_gb300 import _lib as L
    lib = L.load()
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    y = torch.zeros(16, dtype=torch.float32, device="cuda")
    for bad in (0.0, math.nan, math.inf):
        assert lib.mg_cast_fp32(x.data_ptr(), y.data_ptr(), bad, 16, None) == L.MG_ERR_ARG
        assert lib.mg_update_fp64(x.data_ptr(), y.data_ptr(), bad, 16, None) == L.MG_ERR_ARG
    # y inside x's bytes
    assert lib.mg_cast_fp32(x.data_ptr(), x.data_ptr() + 8, 1.0, 16, None) == L.MG_ERR_ARG
    assert lib.mg_cast_fp32(None, None, 1.0, 0, None) == L.MG_OK
