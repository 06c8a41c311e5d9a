"""Shared helpers of the GPU parity tests: the same seeded inputs go to the
CPU oracle and to the CUDA library; results are compared element by element."""
import numpy as np
import torch

from oracle import tpmg as O
from synthetic import make_problem


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    return t.detach().cpu().numpy()


def problem(nlon, nlat, nz, sigma=0.1, seed=7):
    return make_problem(nlon, nlat, nz, sigma, seed)


def handle_for(P, **params):
    from paper_2307_04528_gb300.solver import MGHandle
    params.setdefault("mixed", 1)
    return MGHandle(dev(P["tx"]), dev(P["ty"]), dev(P["tz"]), dev(P["h"]), **params)


def oracle_levels(P, **params):
    p = O.MGParams(**{k: v for k, v in params.items() if k in O.MGParams.__dataclass_fields__})
    return O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], p), p


def rel_inf(a, ref):
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(a - ref)) / den) if den > 0 else float(np.max(np.abs(a)))


def rel_2(a, ref):
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(a - ref) / den) if den > 0 else float(np.linalg.norm(a))
