"""Batched ensemble (persistent kernels over (system level, tile) work lists,
one CUDA graph per precision, autotuned launch shapes) against the oracle and
against single-system solves on the same handles."""
import numpy as np
import pytest
import torch

from gpu_common import dev, host, oracle_levels, problem, rel_2
from oracle import tpmg as O

pytestmark = pytest.mark.gpu

SHAPES = [(32, 16, 8), (64, 32, 16), (48, 24, 9), (96, 46, 12), (128, 64, 6)]


@pytest.fixture(scope="module")
def batch():
    from paper_2307_04528_gb300.solver import MGBatch
    probs = [problem(*shp, sigma=0.1, seed=100 + i) for i, shp in enumerate(SHAPES)]
    systems = [tuple(dev(P[k]) for k in ("tx", "ty", "tz", "h")) for P in probs]
    B = MGBatch(systems, mixed=1)
    return probs, systems, B


def test_tuning_is_sane(batch):
    _, _, B = batch
    t = B.tuning()
    assert t["smooth_block"] in (64, 128)
    assert t["smooth_grid"] > 0 and t["cell_grid"] > 0 and t["vec_grid"] > 0


def test_batched_fp64_matches_oracle_and_single(batch):
    probs, _, B = batch
    bs = [dev(P["b"]) for P in probs]
    xs, infos = B.solve(bs, tol=1e-10, mixed=False)
    for i, P in enumerate(probs):
        assert infos[i]["status"] == 0 and infos[i]["rel_res"] <= 1e-10
        lev, p = oracle_levels(P)
        xr, _, st = O.solve(lev, P["b"], 1e-11, params=p)
        assert rel_2(host(xs[i]), xr) <= 1e-9
        xi, inf1 = B.handle(i).solve(bs[i], tol=1e-10)
        assert abs(inf1["iterations"] - infos[i]["iterations"]) <= 1
        assert rel_2(host(xs[i]), host(xi)) <= 1e-9


def test_batched_mixed_matches_fp64_oracle(batch):
    probs, _, B = batch
    bs = [dev(P["b"]) for P in probs]
    xs, infos = B.solve(bs, tol=1e-10, mixed=True)
    for i, P in enumerate(probs):
        assert infos[i]["status"] == 0 and infos[i]["rel_res"] <= 1e-10
        lev, p = oracle_levels(P)
        xr, _, _ = O.solve(lev, P["b"], 1e-11, params=p)
        assert rel_2(host(xs[i]), xr) <= 1e-9
    # systems converge independently: iteration counts may differ
    assert all(inf["iterations"] >= 1 for inf in infos)


def test_batched_repeat_is_deterministic(batch):
    probs, _, B = batch
    bs = [dev(P["b"]) for P in probs]
    xa, _ = B.solve(bs, tol=1e-8, mixed=True)
    xb, _ = B.solve(bs, tol=1e-8, mixed=True)
    for a, b in zip(xa, xb):
        assert torch.equal(a, b)


def test_batched_large_members_column_paths():
    """Members large enough for the column-walk residual (>= 32768 columns),
    the multi-layer transfers and the single-system kernels of large levels
    (768 x 384 = 294,912 columns), next to a small one: the batched mixed
    solve meets the tolerance on the oracle's own FP64 residual and agrees
    with the single-system mixed solve of each member."""
    from paper_2307_04528_gb300.solver import MGBatch
    shapes = [(256, 192, 12), (768, 384, 4), (64, 32, 16)]
    probs = [problem(*shp, sigma=0.1, seed=300 + i) for i, shp in enumerate(shapes)]
    systems = [tuple(dev(P[k]) for k in ("tx", "ty", "tz", "h")) for P in probs]
    B = MGBatch(systems, mixed=1)
    bs = [dev(P["b"]) for P in probs]
    xs, infos = B.solve(bs, tol=1e-10, mixed=True)
    for i, P in enumerate(probs):
        assert infos[i]["status"] == 0 and infos[i]["rel_res"] <= 1e-10
        lev, _ = oracle_levels(P)
        rel = O.norm2(O.residual(lev[0], P["b"], host(xs[i]))) / O.norm2(P["b"])
        assert rel <= 1e-10 and abs(rel - infos[i]["rel_res"]) <= 1e-12
        xi, _ = B.handle(i).solve_mixed(bs[i], tol=1e-10)
        assert rel_2(host(xs[i]), host(xi)) <= 1e-8
    # the FP64 batched solve takes the same large-level dispatch
    x64, inf64 = B.solve(bs, tol=1e-10, mixed=False)
    for i, P in enumerate(probs):
        assert inf64[i]["status"] == 0 and inf64[i]["rel_res"] <= 1e-10
        lev, _ = oracle_levels(P)
        rel = O.norm2(O.residual(lev[0], P["b"], host(x64[i]))) / O.norm2(P["b"])
        assert rel <= 1e-10 and abs(rel - inf64[i]["rel_res"]) <= 1e-12
        xi, inf1 = B.handle(i).solve(bs[i], tol=1e-10)
        assert abs(inf1["iterations"] - inf64[i]["iterations"]) <= 1
        assert rel_2(host(x64[i]), host(xi)) <= 1e-8


def test_batch_with_an_operational_size_member():
    """A batch whose members include a 1024 x 768 x 70 system (the ensemble's
    third member size: its finest level runs the single-system kernels inside
    the batched steps) next to small ones: mixed solve to 1e-8, each member
    within one FP32 iteration of its single-system solve on the same handle,
    and its residual recomputed by the oracle from the GPU solution."""
    from paper_2307_04528_gb300.solver import MGBatch
    shapes = [(1024, 768, 70), (64, 32, 16), (256, 192, 70)]
    probs = [problem(*shp, sigma=0.1, seed=5100 + i) for i, shp in enumerate(shapes)]
    systems = [tuple(dev(P[k]) for k in ("tx", "ty", "tz", "h")) for P in probs]
    B = MGBatch(systems, mixed=1)
    del systems
    bs = [dev(P["b"]) for P in probs]
    xs, infos = B.solve(bs, tol=1e-8, mixed=True)
    for i, P in enumerate(probs):
        assert infos[i]["status"] == 0 and infos[i]["rel_res"] <= 1e-8
        lev, _ = oracle_levels(P, levels=1)
        rel = O.norm2(O.residual(lev[0], P["b"], host(xs[i]))) / O.norm2(P["b"])
        assert rel <= 1e-8 and abs(rel - infos[i]["rel_res"]) <= 1e-12
        xi, inf1 = B.handle(i).solve_mixed(bs[i], tol=1e-8)
        assert abs(inf1["inner_iterations"] - infos[i]["inner_iterations"]) <= 1
        assert rel_2(host(xs[i]), host(xi)) <= 1e-6
