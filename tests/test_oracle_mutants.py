"""Plant plausible mistakes in a copy of the oracle and check the pins catch them.

Each case copies oracle/*.c|*.h to a temporary directory, applies one textual
edit (a flipped sign, a wrong index, a dropped term, a swapped weight),
compiles it and reruns the pins of tests/test_oracle_pins.py against it.
At least one pin must fail for every mutant.  Nothing here touches the
committed oracle.
"""
import os
import shutil
import subprocess

import pytest

import test_golden_paper as golden
import test_oracle_convergence as conv
import test_oracle_pins as pins
from oracle import build as obuild
from oracle import tpmg as O

MUTANTS = [
    ("east flux sign", "tpmg_oracle_real.h",
     "acc += tx[c] * (uc - u[IX(k, j, ie)]);", "acc -= tx[c] * (uc - u[IX(k, j, ie)]);"),
    ("west face uses own coefficient", "tpmg_oracle_real.h",
     "acc += tx[IX(k, j, iw)] * (uc - u[IX(k, j, iw)]);", "acc += tx[c] * (uc - u[IX(k, j, iw)]);"),
    ("lower vertical flux dropped", "tpmg_oracle_real.h",
     "if (k > 0) acc += tz[IX(k - 1, j, i)] * (uc - u[IX(k - 1, j, i)]);", ""),
    ("south face in the column diagonal dropped", "tpmg_oracle_real.h",
     "if (j > 0) s += ty[IX(k, j - 1, i)];", ""),
    ("forward sweep coupling dropped", "tpmg_oracle_real.h",
     "y[k] = (r[c] + tdn * y[k - 1]) / p[k];", "y[k] = r[c] / p[k];"),
    ("backward sweep uses t/p instead of q/p", "tpmg_oracle_real.h",
     "x[k] = x[k + 1] + (y[k] - (q[k] / p[k]) * x[k + 1]);",
     "x[k] = x[k + 1] + (y[k] - (tz[IX(k, j, i)] / p[k]) * x[k + 1]);"),
    ("smoother sign as printed in Eq. (1)", "tpmg_oracle_real.h",
     "u[c] = (one - omega) * u[c] + omega * x[k];", "u[c] = (one + omega) * u[c] - omega * x[k];"),
    ("smoother right-hand side misses the north neighbour", "tpmg_oracle_real.h",
     "if (j + 1 < nlat) v += ty[c] * u[IX(k, j + 1, i)];", ""),
    ("restriction lon weights swapped", "tpmg_oracle_real.h",
     "bc[base + I] += w * three4 * rv;", "bc[base + I] += w * one4 * rv;"),
    ("prolongation lon neighbour on the wrong side", "tpmg_oracle_real.h",
     "*Inb = (i % 2 == 0) ? (*I + nlon_c - 1) % nlon_c : (*I + 1) % nlon_c;",
     "*Inb = (i % 2 == 1) ? (*I + nlon_c - 1) % nlon_c : (*I + 1) % nlon_c;"),
    ("coarse lon coupling not rescaled", "tpmg_oracle.c",
     "txc[c] *= sx;", "txc[c] *= 1.0;"),
    ("coarse Helmholtz term misses a child", "tpmg_oracle.c",
     "hc[c] += h[f];", "if (i % 2 == 0) hc[c] += h[f];"),
    ("presmoothing residual misses the (1 - omega) factor", "tpmg_oracle_real.h",
     "REAL v = om1 * b[c];", "REAL v = b[c];"),
    ("presmoothing residual misses the north coupling", "tpmg_oracle_real.h",
     "if (j + 1 < nlat) v += ty[IX(k, j, i)] * u[IX(k, j + 1, i)];  /* north */", ""),
    ("gradient face term sign", "tpmg_oracle.c",
     "gtx[c] = -(lam[c] - lam[e]) * (x[c] - x[e]);", "gtx[c] = (lam[c] - lam[e]) * (x[c] - x[e]);"),
]

PINS = [
    pins.test_operator_kills_constants_exactly,
    pins.test_operator_symmetric,
    pins.test_column_solve_matches_exact_rational_solve_of_Hz,
    pins.test_smoother_is_eq1_with_convergent_sign,
    pins.test_coarse_operator_conserves_volume_and_stays_spd,
    pins.test_transfers_adjoint_and_exact_for_linear_fields,
    pins.test_vcycle_symmetric_positive_linear,
    conv.test_one_order_of_magnitude_per_iteration,
    pins.test_gradient_matches_dense_lu_and_finite_differences,
    pins.test_presmooth_residual_is_the_exact_residual_of_the_sweep,
]


def _golden_condition_number():
    golden.test_shallow_multigrid_condition_number((256, 128, 8))


PINS.append(_golden_condition_number)


def test_golden_pin_alone_catches_coarse_assembly_mutants(tmp_path, monkeypatch):
    """The Section 2.3 figures by themselves catch the two coarse-operator
    mutants."""
    for name, fname, old, new in MUTANTS:
        if not name.startswith("coarse"):
            continue
        sub = tmp_path / name.replace(" ", "_")
        sub.mkdir()
        lib = _build_mutant(str(sub), fname, old, new)
        monkeypatch.setattr(O, "_LIB", None)
        monkeypatch.setattr(O._build, "build", lambda force=False, lib=lib: lib)
        with pytest.raises(AssertionError):
            _golden_condition_number()
        monkeypatch.setattr(O, "_LIB", None)


def _build_mutant(tmp, fname, old, new):
    src_dir = os.path.dirname(obuild.SRC[0])
    for f in ("tpmg_oracle.c", "tpmg_oracle_real.h"):
        shutil.copy(os.path.join(src_dir, f), tmp)
    path = os.path.join(tmp, fname)
    text = open(path).read()
    assert text.count(old) == 1, old
    open(path, "w").write(text.replace(old, new))
    lib = os.path.join(tmp, "libmutant.so")
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    "-std=c11", "-o", lib, os.path.join(tmp, "tpmg_oracle.c"), "-lm"],
                   check=True)
    return lib


@pytest.mark.parametrize("name,fname,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(tmp_path, monkeypatch, name, fname, old, new):
    lib = _build_mutant(str(tmp_path), fname, old, new)
    monkeypatch.setattr(O, "_LIB", None)
    monkeypatch.setattr(O._build, "build", lambda force=False: lib)
    caught = []
    for pin in PINS:
        try:
            pin()
        except (AssertionError, Exception) as exc:  # a pin failing in any way counts
            caught.append((pin.__name__, type(exc).__name__))
    monkeypatch.setattr(O, "_LIB", None)
    assert caught, f"no pin caught mutant: {name}"
