"""CPU-side checks of the C ABI: the library builds, loads, exports every
function include/tpmg.h declares, and its host-only entry points (parameter
defaults, workspace sizing, argument validation) behave without a GPU."""
import ctypes
import os
import re
import shutil

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tpmg.h")

pytestmark = pytest.mark.skipif(shutil.which("nvcc") is None and
                                not os.path.exists(os.path.join(
                                    ROOT, "paper_2307_04528_gb300", "_lib", "libtpmg.so")),
                                reason="needs nvcc or a built libtpmg.so")


@pytest.fixture(scope="module")
def lib():
    from paper_2307_04528_gb300 import build
    from paper_2307_04528_gb300 import _lib as L
    build.build()
    return L.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_default_params(lib):
    from paper_2307_04528_gb300 import _lib as L
    p = L.default_params()
    assert (p.levels, p.nu1, p.nu2, p.coarse_iters, p.method, p.mixed) == (0, 1, 1, 12, 0, 0)
    assert p.omega == 0.85 and p.alpha_c == 0.6 and p.maxit == 200 and p.inner_tol == 5e-4
    assert p.inner_maxit == 12 and p.coarse_method == L.MG_COARSE_JACOBI


def _bytes(lib, nlon, nlat, nz, **kw):
    from paper_2307_04528_gb300 import _lib as L
    g = L.mg_grid(nlon, nlat, nz)
    p = L.default_params(**kw)
    n = ctypes.c_size_t(0)
    st = lib.mg_workspace_bytes(ctypes.byref(g), ctypes.byref(p), ctypes.byref(n))
    return st, n.value


def test_workspace_sizing(lib):
    st, n1 = _bytes(lib, 64, 32, 16)
    assert st == 0 and n1 > 64 * 32 * 16 * 8 * 10
    st, n2 = _bytes(lib, 64, 32, 16, mixed=1)
    assert st == 0 and n2 > n1
    st, n3 = _bytes(lib, 1536, 1152, 70, mixed=1)
    assert st == 0
    # about 200 B per fine cell with the FP32 hierarchy, under 30 GB
    cells = 1536 * 1152 * 70
    assert 150 * cells < n3 < 30e9


@pytest.mark.parametrize("shape,kw", [((64, 31, 16), {}),        # odd nlat
                                      ((2, 32, 16), {}),         # nlon < 4
                                      ((64, 32, 0), {}),         # nz < 1
                                      ((64, 32, 300), {}),       # nz > MG_MAX_NZ
                                      ((64, 32, 193), {}),       # nz = MG_MAX_NZ + 1
                                      ((48, 32, 4), {"levels": 6}),  # 48 not divisible by 32
                                      ((64, 32, 4), {"omega": 2.5}),
                                      ((64, 32, 4), {"nu1": 0}),
                                      ((64, 32, 4), {"coarse_method": 3}),
                                      ((64, 32, 4), {"method": 4}),
                                      ((64, 32, 4), {"method": 3, "line_sweeps": 0})])
def test_bad_arguments_rejected_on_host(lib, shape, kw):
    st, _ = _bytes(lib, *shape, **kw)
    assert st == 1
    assert lib.mg_last_error()


def test_pcg_coarse_solve_sizes_and_batch_rejection(lib):
    from paper_2307_04528_gb300 import _lib as L
    st, jac = _bytes(lib, 64, 32, 16, mixed=1)
    st2, pcg = _bytes(lib, 64, 32, 16, mixed=1, coarse_method=L.MG_COARSE_PCG)
    assert st == st2 == 0 and pcg > jac  # two coarsest-level vectors per precision
    g = (L.mg_grid * 1)(L.mg_grid(64, 32, 16))
    p = L.default_params(mixed=1, coarse_method=L.MG_COARSE_PCG)
    n = ctypes.c_size_t(0)
    assert lib.mg_batch_workspace_bytes(1, g, ctypes.byref(p), ctypes.byref(n)) == L.MG_ERR_ARG


def test_level_counts_follow_nlon(lib):
    from paper_2307_04528_gb300 import _lib as L
    # nlon 1536 = 3 * 2^9 -> coarsest nlon 6 after 8 halvings: 9 levels
    st, _ = _bytes(lib, 1536, 1152, 70)
    assert st == 0
    st, _ = _bytes(lib, 1536, 1152, 70, levels=4)
    assert st == 0


def test_batch_workspace_covers_every_system(lib):
    from paper_2307_04528_gb300 import _lib as L
    shapes = [(32, 16, 8), (64, 32, 16), (96, 46, 12)]
    grids = (L.mg_grid * 3)(*(L.mg_grid(*s) for s in shapes))
    p = L.default_params(mixed=1)
    n = ctypes.c_size_t(0)
    assert lib.mg_batch_workspace_bytes(3, grids, ctypes.byref(p), ctypes.byref(n)) == 0
    singles = sum(_bytes(lib, *s, mixed=1)[1] for s in shapes)
    assert n.value > singles
    bad = (L.mg_grid * 1)(L.mg_grid(64, 31, 8))
    assert lib.mg_batch_workspace_bytes(1, bad, ctypes.byref(p), ctypes.byref(n)) == 1


def test_isotropy_rule_sized_for_full_depth(lib):
    st0, n0 = _bytes(lib, 64, 32, 16)
    st1, n1 = _bytes(lib, 64, 32, 16, levels=-1)
    assert st0 == st1 == 0 and n1 >= n0
    st, _ = _bytes(lib, 64, 32, 16, levels=-1, iso_ratio=0.0)
    assert st == 1


def _ns_bytes(lib, nlon, nlat, nz, **kw):
    from paper_2307_04528_gb300 import _lib as L
    kw.setdefault("method", L.MG_METHOD_BICGSTAB)
    g = L.mg_grid(nlon, nlat, nz)
    p = L.default_params(**kw)
    n = ctypes.c_size_t(0)
    st = lib.mg_ns_workspace_bytes(ctypes.byref(g), ctypes.byref(p), ctypes.byref(n))
    return st, n.value


def test_nonsymmetric_workspace_and_parameter_checks(lib):
    """The nonsymmetric hierarchy holds 15 level fields (seven arrays, the
    column sums, two factor pairs, three vectors) plus the right-hand side on
    coarse levels and ten fine solver vectors, and with mixed = 1 their FP32
    copies; it takes the stationary iteration or BiCGStab, the sweep coarse
    solve and a fixed depth."""
    from paper_2307_04528_gb300 import _lib as L
    st, n = _ns_bytes(lib, 64, 32, 16)
    assert st == 0 and n >= 64 * 32 * 16 * 8 * (15 + 10)
    st2, n2 = _ns_bytes(lib, 64, 32, 16, method=L.MG_METHOD_STATIONARY)
    assert st2 == 0 and n2 == n
    # mixed precision adds the FP32 copies: 12 arrays and 4 vectors per level, 10 fine vectors
    st3, n3 = _ns_bytes(lib, 64, 32, 16, mixed=1)
    assert st3 == 0 and n3 - n >= 64 * 32 * 16 * 4 * (16 + 10)
    for kw in ({"method": L.MG_METHOD_CG}, {"method": L.MG_METHOD_BICGSTAB_LINE},
               {"coarse_method": L.MG_COARSE_PCG}, {"levels": -1}, {"omega": 2.5},
               {"mixed": 1, "inner_maxit": 0}):
        st, _ = _ns_bytes(lib, 64, 32, 16, **kw)
        assert st == L.MG_ERR_ARG, kw
        assert lib.mg_last_error()
    g = L.mg_grid(64, 32, 16)
    p = L.default_params(method=L.MG_METHOD_BICGSTAB)
    h = ctypes.c_void_p()
    co = L.mg_ns_coeffs(0, 0, 0, 0, 0, 0, 0)
    assert lib.mg_ns_setup(ctypes.byref(g), ctypes.byref(co), ctypes.byref(p), None, 0, None,
                           ctypes.byref(h)) == L.MG_ERR_ARG and not h.value
    assert lib.mg_ns_num_levels(None) == 0
