#!/usr/bin/env python
"""Benchmark: milliseconds to a 1e-10 relative residual on the operational-size
lat-lon grid (1536 x 1152 x 70, ~124M unknowns), FP32 multigrid inside FP64
refinement (the headline `value`) next to the plain FP64 multigrid solve.

One step = one solve of H x = b from x = 0 (all kernels of the path).  Inputs
are synthetic (seeded generator of `synthetic`), resident in HBM when the
timed region starts; every array exceeds the 129 MB L2, so no flush is
needed.  N > 1 GPUs run independent replicas (one system per rank, seeds
differ), so scaling is weak and there is no collective on the data path.

`--impl reference` times the CPU oracle instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from synthetic import WORKLOADS, make_ns_problem, make_problem, workload_seed  # noqa: E402
from synthetic.latlon import ENSEMBLE_MEMBERS  # noqa: E402

METRIC = "ms to 1e-10 rel residual, 1536x1152x70: FP32-MG+FP64 refine vs FP64 MG; HBM %"
UNIT = "ms"
TOL = 1e-10


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="latlon_1536x1152x70")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the nonsymmetric and ensemble comparisons after the headline")
    ap.add_argument("--no-paper", action="store_true",
                    help="skip the one-off solves of the paper's own configuration")
    ap.add_argument("--profile-out", default=None,
                    help="write per-(kernel, level, precision) event times of the profiled "
                         "repeat to this JSON file")
    ap.add_argument("--kernel", choices=sorted(PROBE_KERNELS), default=None,
                    help="time one kernel (or one solve) in isolation on --shape instead of "
                         "the benchmark; the mode the committed ncu summaries run")
    ap.add_argument("--shape", type=int, nargs=3, default=[512, 384, 70],
                    metavar=("NLON", "NLAT", "NZ"))
    ap.add_argument("--launches", type=int, default=5)
    ap.add_argument("--sigma", type=float, default=0.2)
    ap.add_argument("--krylov-maxit", type=int, default=8000,
                    help="iteration cap of the line-relaxed BiCGStab in --workload krylov")
    return ap.parse_args()


from paper_2307_04528_gb300.replicas import dist_env  # noqa: E402


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------- CPU oracle
def oracle_setup(P):
    """The oracle's hierarchy and its FP32 copies (setup, untimed, as the
    GPU's mg_setup is untimed)."""
    from oracle import tpmg as O
    p = O.MGParams()
    lev = O.build_hierarchy(P["tx"], P["ty"], P["tz"], P["h"], p)
    return lev, O.float_levels(lev), p


def oracle_solve_ms(P, lev, l32, p, mixed: bool):
    """One complete solve of the oracle from x = 0 to ||b - H x|| <= 1e-10 ||b||
    on the host cores, wall-clock timed: the mixed-precision solve (FP32
    V-cycles inside FP64 refinement) or the FP64 solve.  Returns (ms, outer
    iterations, status)."""
    from oracle import tpmg as O
    t0 = time.perf_counter()
    if mixed:
        _, hist, st = O.solve_mixed(lev, P["b"], TOL, params=p, levels32=l32)
    else:
        _, hist, st = O.solve(lev, P["b"], TOL, params=p)
    return (time.perf_counter() - t0) * 1e3, len(hist) - 1, int(st)


def run_reference(args):
    """The oracle's mixed-precision solve of the workload, timed on the host
    cores.  A complete solve takes ~30 s there, so a step is one of its
    refinement steps, in rotation: step s runs refinement step k = s mod m
    (m of them to 1e-10) from the iterate the oracle's own solve had entering
    it (prepared untimed), i.e. the FP64 residual, its norm, the FP32 inner
    solve and the FP64 update, plus, for the last one, the final residual
    and stopping test.  The m step kinds add up to exactly the work of one
    solve, so `value` = the sum over k of the mean time of step kind k (a
    solve assembled from measured parts, no extrapolation) and ms_per_step
    is the mean time of one step.  The W warm-up steps are one oracle FP32
    V-cycle each (pages every level in and starts the thread pool)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import tpmg as O
    w = WORKLOADS[args.workload]
    P = make_problem(w["nlon"], w["nlat"], w["nz"], w["sigma"], workload_seed(args.workload))
    lev, l32, p = oracle_setup(P)
    b = P["b"]
    bn = O.norm2(b)
    starts = [np.zeros_like(b)]
    _, hist, st = O.solve_mixed(lev, b, TOL, params=p, levels32=l32,
                                track=lambda x: starts.append(x.copy()))
    m = len(hist) - 1
    if st != O.OK or m < 1:
        raise RuntimeError(f"oracle mixed solve status {st} after {m} refinement steps")
    r32 = (b / np.max(np.abs(b))).astype(np.float32)
    for _ in range(args.warmup):
        O.vcycle(l32, r32, p)
    times = [[] for _ in range(m)]
    final = None
    for step in range(args.steps):
        k = step % m
        x = starts[k].copy()
        t0 = time.perf_counter()
        r = O.residual(lev[0], b, x)
        rn = O.norm2(r)
        O.refine_correct(l32, x, r, rn, bn, TOL, p)
        if k == m - 1:
            final = O.norm2(O.residual(lev[0], b, x)) / bn
        times[k].append((time.perf_counter() - t0) * 1e3)
    done = [t for t in times if t]
    if len(done) < m:
        raise RuntimeError(f"--steps {args.steps} < {m} refinement steps: no complete solve")
    v = sum(statistics.mean(t) for t in times)
    per_step = statistics.mean(t for ts in times for t in ts)
    out = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "tol": TOL, "refinement_steps": m,
                   "step": "one refinement step of the oracle's mixed solve, in rotation",
                   "step_ms_by_refinement_step": [statistics.mean(t) for t in times],
                   "final_rel_res": final, "oracle_status": int(st),
                   "warmup": "one oracle FP32 V-cycle per warm-up step"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"the oracle's mixed-precision solve at {args.workload} to "
                                   f"1e-10 from x = 0, its {m} refinement steps timed one per "
                                   f"step in rotation and summed (wall clock)"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


# ----------------------------------------------------------------- GPU arm
# algorithmic words moved per fine cell by each fine-level kernel class
# (reads + writes of distinct arrays; horizontal neighbours counted once)
KERNEL_WORDS = {
    # (kind, prec): (name, words per cell)
    (0, 1): ("smooth fp32 (+ <r, z>)", 8),            # u b tx ty tz m dq -> u
    (1, 1): ("smooth fp32 zero guess", 5),            # b tz m dq -> u
    (2, 1): ("residual + restriction fp32", 6),       # u b tx ty tz h -> b_c (+ coarse write;
                                                      # u b tx ty after a sweep from zero)
    (3, 1): ("direction update + apply fp32", 8),     # z d tx ty tz h -> d q
    (5, 1): ("prolongation + correction fp32", 2),    # u e_c -> u (+ coarse read)
    (0, 0): ("smooth fp64", 8),                       # u b tx ty tz m dq -> u
    (1, 0): ("smooth fp64 zero guess", 5),
    (2, 0): ("residual fp64 -> scaled fp32", 6.5),    # x b tx ty tz h -> r32
    (3, 0): ("apply fp64", 6),
}


# DRAM bytes per fine cell of one k_smooth_dot<float> launch (ncu capture at
# 512x384x70: 397.3 MB read + 34.8 MB written for 13,762,560 cells)
SMOOTH_DOT_DRAM_BYTES_PER_CELL = (397.266944e6 + 34.799616e6) / (512 * 384 * 70)
# DRAM bytes per fine cell of one k_resid_restrict<float> launch in its
# presmoothing form on the finest level (ncu capture at 512x384x70: 232.6 MB
# read + 16.1 MB written for 13,762,560 fine cells)
RESID_RESTRICT_PRE_DRAM_BYTES_PER_CELL = (232.561408e6 + 16.097536e6) / (512 * 384 * 70)


def kernel_table(H, L, N):
    rows = []
    c = H.level_shape(1) if H.num_levels > 1 else (0, 0, 0)
    coarse_ratio = c[0] * c[1] * c[2] / N  # level-1 cells per fine cell
    for (kind, prec), (name, words) in KERNEL_WORDS.items():
        n, ms = H.profile_read(kind, 0, prec)
        if n == 0:
            continue
        if (kind, prec) == (2, 1) and H.params.nu1 == 1:
            words = 4  # the presmoothing form reads u, b, tx, ty
        if (kind, prec) in ((2, 1), (5, 1)):
            words = words + coarse_ratio
        avg = ms / n
        nbytes = words * (4 if prec == 1 else 8) * N
        rows.append({"kernel": name, "launches": n, "avg_ms": round(avg, 4),
                     "alg_bytes": nbytes, "gbs": round(nbytes / (avg * 1e-3) / 1e9, 1)})
    return rows


# the paper's configuration: (label, mg_params overrides, mixed, maxit cap)
PAPER_RUNS = [
    ("stationary_default_hierarchy_fp64", dict(method=1), False, 200),
    ("stationary_default_hierarchy_mixed", dict(method=1, inner_maxit=40), True, 40),
    ("stationary_4_levels_fp64", dict(method=1, levels=4), False, 60),
    ("cg_4_levels_mixed", dict(levels=4, inner_maxit=40), True, 40),
    ("cg_4_levels_chebyshev24_mixed", dict(levels=4, inner_maxit=40, coarse_method=2,
                                           coarse_iters=24), True, 40),
    ("cg_4_levels_pcg24_mixed", dict(levels=4, inner_maxit=40, coarse_method=1,
                                     coarse_iters=24), True, 40),
]


def paper_config(MGHandle, coeffs, b, barrier):
    """Time one solve of each PAPER_RUNS entry to 1e-10 (or its iteration cap)
    with CUDA events, on a handle built for it; returns a dict of times,
    iteration counts, the residual reached and the mean residual reduction per
    outer FP64 iteration (the quantity Section 2 puts near 0.1)."""
    import torch
    out = {}
    stream = torch.cuda.current_stream()
    for label, over, mixed, cap in PAPER_RUNS:
        Hp = MGHandle(*coeffs, mixed=int(mixed), maxit=cap, **over)
        x = torch.zeros_like(b)
        fn = Hp.solve_mixed if mixed else Hp.solve
        fn(b, x, tol=TOL, raise_on_error=False)  # warm-up (captures the V-cycle graph)
        x.zero_()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        _, info = fn(b, x, tol=TOL, raise_on_error=False)
        ev1.record(stream)
        barrier()
        hist = info["history"]
        its = max(len(hist) - 1, 1)
        out[label] = {"ms": ev0.elapsed_time(ev1), "status": info["status"],
                      "iterations": info["iterations"],
                      "fp32_iterations": info["inner_iterations"] if mixed else None,
                      "rel_res": info["rel_res"], "levels": Hp.num_levels,
                      "reduction_per_iteration": (hist[-1] / hist[0]) ** (1.0 / its)
                      if hist and hist[0] > 0 else None}
        del Hp, x
        torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    from paper_2307_04528_gb300 import replicas
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    replicas.init()
    from paper_2307_04528_gb300 import _lib as L
    from paper_2307_04528_gb300.solver import MGHandle

    w = WORKLOADS[args.workload]
    # replicas only: every rank solves its own system (seed + rank)
    P = make_problem(w["nlon"], w["nlat"], w["nz"], w["sigma"],
                     replicas.replica_seed(workload_seed(args.workload), rank))
    N = P["h"].size
    d = lambda a: torch.as_tensor(a, dtype=torch.float64).cuda()
    tx, ty, tz, hh, b = d(P["tx"]), d(P["ty"]), d(P["tz"]), d(P["h"]), d(P["b"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    H = MGHandle(tx, ty, tz, hh, mixed=1)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    x = torch.zeros_like(b)
    lib = L.load()
    stream = torch.cuda.current_stream()

    def barrier():
        replicas.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):
        return replicas.max_over_ranks(v, device="cuda")

    def timed(fn, steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        infos = [fn() for _ in range(steps)]
        ev1.record(stream)
        barrier()
        return ev0.elapsed_time(ev1), infos

    def mixed_step():
        x.zero_()
        _, info = H.solve_mixed(b, x, tol=TOL)
        return info

    def fp64_step():
        x.zero_()
        _, info = H.solve(b, x, tol=TOL)
        return info

    for _ in range(args.warmup):
        mixed_step()
    fp64_step()

    # headline: mixed precision, clocks sampled during the timed region
    clocks = ClockSampler(local)
    n0 = lib.mg_launch_count()
    ms_mixed, infos = timed(mixed_step, args.steps)
    launches = lib.mg_launch_count() - n0
    clk = clocks.stop()
    ms_mixed = max_over_ranks(ms_mixed / args.steps)
    info_m = infos[-1]
    # end to end through the public API with host buffers (pinned), right
    # after the device-resident steps (before the FP64 comparison solves)
    e2e = None
    if not args.no_e2e:
        hb = torch.from_numpy(P["b"]).pin_memory()
        hx = torch.empty_like(hb).pin_memory()

        def e2e_step():
            bd = hb.to("cuda", non_blocking=True)
            xd = torch.zeros_like(bd)
            _, info = H.solve_mixed(bd, xd, tol=TOL)
            hx.copy_(xd, non_blocking=True)
            return info

        e2e_step()
        ms_e2e, _ = timed(e2e_step, args.steps)
        ms_e2e = max_over_ranks(ms_e2e / args.steps)
        e2e = {"value": ms_e2e, "unit": UNIT, "h2d_bytes_per_step": int(hb.numel() * 8),
               "d2h_bytes_per_step": int(hx.numel() * 8)}

    # the same timed steps again with CUDA events around every launch
    H.profile(2)  # events around every launch of every level
    ms_prof, _ = timed(mixed_step, args.steps)
    sm_calls, sm_ms = H.profile_read(L.K_SMOOTH, 0, L.MG_PREC_FP32)
    rr_calls, rr_ms = H.profile_read(L.K_RESID, 0, L.MG_PREC_FP32)
    rr_all = [H.profile_read(L.K_RESID, lvl, L.MG_PREC_FP32) for lvl in range(H.num_levels)]
    res_calls, res_ms = H.profile_read(L.K_RESID, 0, L.MG_PREC_FP64)
    kernels = kernel_table(H, L, N)
    if args.profile_out:
        full = []
        for lvl in range(H.num_levels):
            for kind in range(7):
                for prec in (0, 1):
                    n, ms = H.profile_read(kind, lvl, prec)
                    if n:
                        full.append({"kind": kind, "level": lvl, "prec": prec, "launches": n,
                                     "total_ms": ms, "avg_us": 1e3 * ms / n,
                                     "shape": H.level_shape(lvl)})
        with open(args.profile_out, "w") as f:
            json.dump({"steps": args.steps, "ms_per_step_profiled": None, "rows": full}, f,
                      indent=1)
    H.profile(False)
    ms_prof = max_over_ranks(ms_prof / args.steps)

    ms_fp64, infos64 = timed(fp64_step, args.steps)
    ms_fp64 = max_over_ranks(ms_fp64 / args.steps)
    info_d = infos64[-1]

    # the paper's own configuration, each solve timed once: the stationary
    # iteration x <- x + V(b - H x) (Section 2) on the default hierarchy, and
    # on the 4-level shallow hierarchy of Section 2.3 (capped: its iteration
    # count grows with resolution), beside the CG-accelerated default
    paper = paper_config(MGHandle, (tx, ty, tz, hh), b, barrier) if not args.no_paper else None
    del tx, ty, tz, hh

    peak, peak_kind = load_peaks()
    # the kernel with the largest share of the mixed solve: the V-cycle's last
    # fine-level sweep with <r, z> fused (reads u, b, tx, ty, tz, m, dq; writes
    # u: 8 x 4 B per cell)
    sm_bytes = 32 * N
    sm_avg_ms = sm_ms / max(sm_calls, 1)
    achieved = sm_bytes / (sm_avg_ms * 1e-3) / 1e9 if sm_calls else None
    roofline = {"kernel": "k_smooth_dot<float>: fine-level block-Jacobi sweep of Eq. (1) "
                          "(last sweep of the V-cycle, CG inner product fused)", "bound": "hbm",
                "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": SMOOTH_DOT_DRAM_BYTES_PER_CELL * N,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch at "
                                  "512x384x70, scaled per cell to this grid",
                "launches_timed": sm_calls, "avg_ms": sm_avg_ms,
                "bytes_per_launch": sm_bytes, "peak_source": peak_kind,
                "share_of_step": (sm_ms / args.steps) / ms_prof if ms_prof else None,
                "timed_region": "repeat of the K timed mixed solves with events around "
                                "every launch", "ms_per_step_profiled": ms_prof}
    # the next kernel: the FP32 V-cycle's residual and restriction in one pass,
    # finest-level launches.  After the single pre-smoothing sweep from zero it
    # reads u, b, tx, ty (the presmoothing form); otherwise also tz and h.
    # Both write the coarse right-hand side (level-1 cells).
    c1 = H.level_shape(1) if H.num_levels > 1 else (0, 0, 0)
    pre = H.params.nu1 == 1
    rr_bytes = 4 * ((4 if pre else 6) * N + c1[0] * c1[1] * c1[2])
    rr_avg_ms = rr_ms / max(rr_calls, 1)
    rr_gbs = rr_bytes / (rr_avg_ms * 1e-3) / 1e9 if rr_calls else None
    rr_cells = RESID_RESTRICT_PRE_DRAM_BYTES_PER_CELL if pre else None
    ms_rr_all = sum(ms for _, ms in rr_all)
    roofline_next = {"kernel": "k_resid_restrict<float>: residual and its restriction R = P^T in "
                               "one pass (" + ("presmoothing form" if pre else "full stencil") +
                               "), finest-level launches", "achieved": rr_gbs, "unit": "GB/s",
                     "frac": (rr_gbs / peak) if rr_gbs else None,
                     "traffic": rr_cells * N if rr_cells is not None else None,
                     "launches_timed": rr_calls, "avg_ms": rr_avg_ms,
                     "bytes_per_launch": rr_bytes,
                     "share_of_step_all_levels": (ms_rr_all / args.steps) / ms_prof
                     if ms_prof else None}
    res_avg = res_ms / max(res_calls, 1)

    out = {
        "metric": METRIC, "value": ms_mixed, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mixed, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": args.workload, "unknowns": int(N), "tol": TOL,
                   "parallelism": f"replicas{world}", "l2": "inputs larger than L2 (no flush)",
                   "mixed_refinement_steps": info_m["iterations"],
                   "mixed_fp32_iterations": info_m["inner_iterations"],
                   "mixed_rel_res": info_m["rel_res"],
                   "fp64_ms": ms_fp64, "fp64_iterations": info_d["iterations"],
                   "fp64_rel_res": info_d["rel_res"],
                   "speedup_mixed_vs_fp64": ms_fp64 / ms_mixed,
                   "levels": H.num_levels, "setup_ms": setup_ms,
                   "fp64_residual_kernel_avg_ms": res_avg,
                   "paper_configuration": paper},
        "gpu_launches": int(launches),
        "kernels_fine_level": kernels,
        "clocks": clk,
        "roofline": roofline,
        "roofline_next": roofline_next,
    }
    if e2e:
        out["e2e"] = e2e
    if rank == 0 and world == 1 and not args.no_extra:
        # the other comparisons, after every headline measurement, on the
        # memory the headline handle leaves
        del H, x, b, lib
        torch.cuda.empty_cache()
        for key, fn in (("nonsymmetric_transport", lambda: ns_measure(min(args.steps, 3))),
                        ("ensemble_24", lambda: ensemble_measure(min(args.steps, 3), 1))):
            try:
                out[key] = fn()
            except Exception as exc:  # reported, never fatal to the headline line
                out[key] = {"error": f"{type(exc).__name__}: {exc}"}
                torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import tpmg as O
        lev, l32, p = oracle_setup(P)
        ms, its, st = oracle_solve_ms(P, lev, l32, p, mixed=True)
        out["cpu_baseline"] = {
            "value": ms, "unit": UNIT, "cores": O.num_threads(), "kind": "oracle",
            "sample": f"one complete mixed-precision solve of the oracle at {args.workload} to "
                      f"1e-10 from x = 0, timed (wall clock)",
            "refinement_steps": its, "status": st}
    if rank == 0:
        print(json.dumps(out))
    replicas.finalize()


# ----------------------------------------------------------------- ensemble
def _gen_member(task):
    nlon, nlat, nz, seed = task
    P = make_problem(nlon, nlat, nz, 0.1, seed)
    return {k: P[k] for k in ("tx", "ty", "tz", "h", "b")}


def run_ensemble(args):
    """The ensemble comparison as its own JSON line (ensemble_measure)."""
    print(json.dumps(ensemble_measure(args.steps, args.warmup)))


def ensemble_measure(steps, warmup):
    """24 independent systems of uneven sizes (8 at 256x192x70, 8 at 512x384x70,
    6 at 1024x768x70, 2 at 1536x1152x70), FP32 MG inside FP64 refinement to
    1e-8: one batched solve (persistent kernels, one CUDA graph) against the
    same systems solved one after another on the same hierarchies."""
    import multiprocessing as mp

    import torch
    from paper_2307_04528_gb300 import _lib as L
    from paper_2307_04528_gb300.solver import MGBatch

    tol = 1e-8
    tasks = []
    for count, nlon, nlat, nz in ENSEMBLE_MEMBERS:
        for _ in range(count):
            tasks.append((nlon, nlat, nz, workload_seed("ensemble", len(tasks))))
    systems, bs = [], []
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(8, os.cpu_count() or 1)) as pool:
        for P in pool.imap(_gen_member, tasks):
            systems.append(tuple(torch.as_tensor(P[k]).cuda() for k in ("tx", "ty", "tz", "h")))
            bs.append(torch.as_tensor(P["b"]).cuda())
            del P
    cells = sum(b.numel() for b in bs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B = MGBatch(systems, mixed=1)
    torch.cuda.synchronize()
    setup_ms = (time.perf_counter() - t0) * 1e3
    del systems
    torch.cuda.empty_cache()
    xs = [torch.zeros_like(b) for b in bs]
    lib = L.load()
    stream = torch.cuda.current_stream()

    def batched():
        for x in xs:
            x.zero_()
        _, infos = B.solve(bs, xs, tol=tol, mixed=True)
        return infos

    handles = [B.handle(i) for i in range(len(bs))]

    def sequential():
        infos = []
        for i, H in enumerate(handles):
            xs[i].zero_()
            _, info = H.solve_mixed(bs[i], xs[i], tol=tol)
            infos.append(info)
        return infos

    def timed(fn, steps):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        out = [fn() for _ in range(steps)]
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1) / steps, out[-1]

    for _ in range(warmup):
        batched()
    sequential()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    n0 = lib.mg_launch_count()
    ms_b, infos_b = timed(batched, steps)
    launches = lib.mg_launch_count() - n0
    clk = clocks.stop()
    ms_s, infos_s = timed(sequential, steps)
    out = {
        "metric": "ms per ensemble solve to 1e-8 rel residual, 24 uneven lat-lon systems "
                  "(FP32-MG+FP64 refine), batched vs sequential",
        "value": ms_b, "unit": "ms", "n_gpus": 1, "steps": steps, "warmup": warmup,
        "ms_per_step": ms_b, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "ensemble_24", "members": [list(t[:3]) for t in tasks],
                   "unknowns": int(cells), "tol": tol, "sequential_ms": ms_s,
                   "speedup_batched_vs_sequential": ms_s / ms_b, "setup_ms": setup_ms,
                   "tuning": B.tuning(),
                   "refinement_steps": [i["iterations"] for i in infos_b],
                   "fp32_iterations": [i["inner_iterations"] for i in infos_b],
                   "max_rel_res": max(i["rel_res"] for i in infos_b),
                   "sequential_max_rel_res": max(i["rel_res"] for i in infos_s),
                   "sequential_fp32_iterations": [i["inner_iterations"] for i in infos_s]},
        "gpu_launches": int(launches), "clocks": clk,
    }
    del B, bs, xs, handles
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------- one kernel
# --kernel name -> (precision, what runs, algorithmic words per fine cell or None)
PROBE_KERNELS = {
    "smooth32": (1, "smooth", 8),
    "smooth32_dot": (1, "smooth_dot", 8),
    "smooth32_zero": (1, "smooth0", 5),
    "resid32": (1, "residual", 7),
    "apply32": (1, "apply", 6),
    "restrict32": (1, "restrict", None),
    "resid_restrict32": (1, "resid_restrict", None),
    "presmooth_restrict32": (1, "presmooth_restrict", None),
    "prolong32": (1, "prolong", None),
    "coarse32": (1, "coarse", None),
    "dir_apply32": (1, "dir_apply", 8),
    "vcycle32": (1, "vcycle", None),
    "smooth64": (0, "smooth", 8),
    "smooth64_zero": (0, "smooth0", 5),
    "resid64": (0, "residual", 7),
    "apply64": (0, "apply", 6),
    "coarse64": (0, "coarse", None),
    "vcycle64": (0, "vcycle", None),
    "coeff_grad64": (0, "coeff_grad", 10),
    # whole solves (ncu picks the kernels of interest by name: the CG vector
    # kernels, the fused direction update + apply, the FP64 refinement residual)
    "solve_mixed": (1, "solve_mixed", None),
    "solve64": (0, "solve", None),
    # a batch of three systems (--shape, half and quarter of it in longitude
    # and latitude), FP32 multigrid in FP64 refinement to 1e-8 (the batched
    # persistent kernels)
    "batch_mixed": (1, "batch", None),
    # the nonsymmetric operator (synthetic transport, pe 0.3), FP64: the
    # apply of H and the transposed-stencil apply of H^T (h, 6 couplings, x ->
    # y), the sweep (b u e w n s d m dq -> u) and the sweep from zero (b d m dq
    # -> u), the V-cycle and BiCGStab solves of H and H^T
    "ns_apply64": (0, "ns_apply", 9),
    "ns_apply64_T": (0, "ns_apply_T", 9),
    "ns_smooth64": (0, "ns_smooth", 10),
    "ns_smooth64_zero": (0, "ns_smooth0", 5),
    "ns_vcycle64": (0, "ns_vcycle", None),
    "ns_smooth32": (1, "ns_smooth", 10),
    "ns_smooth32_zero": (1, "ns_smooth0", 5),
    "ns_vcycle32": (1, "ns_vcycle", None),
    "ns_solve_mixed": (1, "ns_solve_mixed", None),
    "ns_solve64": (0, "ns_solve", None),
    "ns_solve64_T": (0, "ns_solve_T", None),
}


def run_kernel(args):
    """Run one fine-level kernel of the multigrid `--launches` times on a
    seeded system of `--shape` through the library's per-level C ABI and
    print its mean event time (and algorithmic GB/s where the bytes are
    known).  Small cases (a few GB on the device, every array above the
    129 MB L2) are what the ncu captures of the profiles run."""
    import torch

    from paper_2307_04528_gb300.solver import MGHandle

    nlon, nlat, nz = args.shape
    prec, op, words = PROBE_KERNELS[args.kernel]
    d = lambda a, dt=torch.float64: torch.as_tensor(a).to("cuda", dt)
    if op.startswith("ns_"):
        from paper_2307_04528_gb300.solver import NSHandle
        P = make_ns_problem(nlon, nlat, nz, args.sigma, 3000)
        H = NSHandle(*(d(P[k]) for k in ("h", "tx", "ty", "tz", "txr", "tyr", "tzr")), mixed=1)
    else:
        P = make_problem(nlon, nlat, nz, args.sigma, 3000)
        H = MGHandle(d(P["tx"]), d(P["ty"]), d(P["tz"]), d(P["h"]), mixed=1)
    if op == "batch":
        from paper_2307_04528_gb300.solver import MGBatch
        probs = [P] + [make_problem(nlon // f, nlat // f, nz, args.sigma, 3000 + f) for f in (2, 4)]
        B = MGBatch([tuple(d(Q[k]) for k in ("tx", "ty", "tz", "h")) for Q in probs], mixed=1)
        bs = [d(Q["b"]) for Q in probs]
        xs = [torch.zeros_like(bb) for bb in bs]
    dt = torch.float32 if prec == 1 else torch.float64
    gen = torch.Generator(device="cuda").manual_seed(0)
    shape = (nz, nlat, nlon)
    b = torch.randn(shape, generator=gen, device="cuda", dtype=dt)
    u = torch.randn(shape, generator=gen, device="cuda", dtype=dt)
    cshape = H.level_shape(1) if H.num_levels > 1 else shape
    ec = torch.randn(cshape, generator=gen, device="cuda", dtype=dt)
    lshape = H.level_shape(H.num_levels - 1)
    bcoarse = torch.randn(lshape, generator=gen, device="cuda", dtype=dt)
    b64 = d(P["b"])
    x64 = torch.zeros_like(b64)

    def run():
        if op in ("ns_apply", "ns_apply_T"):
            return H.apply(u, transpose=op.endswith("_T"))
        if op == "ns_smooth":
            return H.level_smooth(0, b, u, prec=prec)
        if op == "ns_smooth0":
            return H.level_smooth(0, b, None, prec=prec)
        if op == "ns_vcycle":
            return H.vcycle(b, prec=prec)
        if op in ("ns_solve", "ns_solve_T"):
            x64.zero_()
            return H.solve(b64, x64, tol=TOL, transpose=op.endswith("_T"))
        if op == "ns_solve_mixed":
            x64.zero_()
            return H.solve_mixed(b64, x64, tol=TOL)
        if op == "smooth":
            return H.level_smooth(0, b, u, prec=prec)
        if op == "smooth_dot":
            return H.level_smooth_dot(0, b, u, prec=prec)
        if op == "smooth0":
            return H.level_smooth(0, b, None, prec=prec)
        if op == "residual":
            return H.level_residual(0, b, u, prec=prec)
        if op == "apply":
            return H.level_apply(0, u, prec=prec)
        if op == "restrict":
            return H.level_restrict(0, u, prec=prec)
        if op == "resid_restrict":
            return H.level_residual_restrict(0, b, u, prec=prec)
        if op == "presmooth_restrict":
            return H.level_presmooth_restrict(0, b, u, prec=prec)
        if op == "coarse":
            return H.coarse_solve(bcoarse, prec=prec)
        if op == "vcycle":
            return H.vcycle(b, prec=prec)
        if op == "coeff_grad":
            return H.coeff_grad(b, u)
        if op == "dir_apply":
            return H.level_dir_apply(0, b, u, 0.5, prec=prec)
        if op == "solve_mixed":
            x64.zero_()
            return H.solve_mixed(b64, x64, tol=TOL)
        if op == "solve":
            x64.zero_()
            return H.solve(b64, x64, tol=TOL)
        if op == "batch":
            for xx in xs:
                xx.zero_()
            return B.solve(bs, xs, tol=1e-8, mixed=True)
        return H.level_prolong_add(0, ec, u, prec=prec)

    run()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record()
    for _ in range(args.launches):
        run()
    ev[1].record()
    torch.cuda.synchronize()
    ms = ev[0].elapsed_time(ev[1]) / args.launches
    n = nz * nlat * nlon
    out = {"kernel": args.kernel, "shape": args.shape, "avg_ms": ms}
    if op in ("resid_restrict", "presmooth_restrict"):  # 6 (4) fine arrays read, coarse written
        words = (6 if op == "resid_restrict" else 4) + cshape[0] * cshape[1] * cshape[2] / n
    if op == "restrict":
        words = 1 + cshape[0] * cshape[1] * cshape[2] / n
    if op == "prolong":
        words = 2 + cshape[0] * cshape[1] * cshape[2] / n
    if words:
        nbytes = words * (4 if prec == 1 else 8) * n
        out.update(alg_bytes=nbytes, gbs=nbytes / (ms * 1e-3) / 1e9)
    print(json.dumps(out))


# ----------------------------------------------------------------- Krylov comparison
def run_krylov(args):
    """The paper's comparison (Section 1): the BiCGStab solver preconditioned
    by vertical line relaxation that the multigrid replaced, against the
    multigrid, on this GPU.

    1536 x 1152 x 70 (the operational-size workload), FP64 to 1e-10: BiCGStab
    with one sweep of Eq. (1) as preconditioner (capped at --krylov-maxit
    iterations), BiCGStab and CG preconditioned by the V-cycle.  Beside the
    paper's "about twice as fast" (Section 1; Table 1's solver times
    17.6 vs 26.4 min on 4608 cores, a whole-model run on CPUs).

    1024 x 768 x 70, single precision (Section 1: Krylov solvers run in
    single precision can stall at tight tolerances): each method's whole
    solve in FP32 (mg_solve_single) to an unreachable 1e-10, with its
    residual history, best residual and the error of its final iterate
    against the FP64 multigrid solution; and the mixed-precision refinement
    to 1e-10 with each method as the FP32 inner solver."""
    import torch

    from paper_2307_04528_gb300 import _lib as L
    from paper_2307_04528_gb300.solver import MGHandle

    stream = torch.cuda.current_stream()

    def timed(fn):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        out = fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1), out

    def system(name):
        w = WORKLOADS[name]
        P = make_problem(w["nlon"], w["nlat"], w["nz"], w["sigma"], workload_seed(name))
        d = lambda a: torch.as_tensor(a, dtype=torch.float64).cuda()
        return tuple(d(P[k]) for k in ("tx", "ty", "tz", "h")), d(P["b"])

    out = {"metric": "ms to 1e-10 rel residual: BiCGStab + line relaxation (Section 1) vs "
                     "multigrid; single-precision behaviour", "unit": "ms", "n_gpus": 1,
           "data": "synthetic"}
    methods = {"bicgstab_line": L.MG_METHOD_BICGSTAB_LINE, "bicgstab_mg": L.MG_METHOD_BICGSTAB,
               "cg_mg": L.MG_METHOD_CG, "stationary_mg": L.MG_METHOD_STATIONARY}
    # ---- FP64 at the operational size
    coeffs, b = system("latlon_1536x1152x70")
    fp64 = {}
    for name in ("cg_mg", "bicgstab_mg", "bicgstab_line"):
        cap = args.krylov_maxit if name == "bicgstab_line" else 200
        H = MGHandle(*coeffs, method=methods[name], maxit=cap)
        x = torch.zeros_like(b)
        if name != "bicgstab_line":  # warm-up: the V-cycle graphs are captured on first use
            H.solve(b, x, tol=TOL, raise_on_error=False, history_cap=cap + 64)
            x.zero_()
        ms, (_, info) = timed(lambda: H.solve(b, x, tol=TOL, raise_on_error=False,
                                               history_cap=cap + 64))
        fp64[name] = {"ms": ms, "status": info["status"], "iterations": info["iterations"],
                      "rel_res": info["rel_res"], "ms_per_iteration": ms / max(info["iterations"], 1)}
        del H, x
        torch.cuda.empty_cache()
    fp64["speedup_multigrid_vs_bicgstab_line"] = fp64["bicgstab_line"]["ms"] / fp64["cg_mg"]["ms"]
    out["latlon_1536x1152x70_fp64"] = fp64
    del coeffs, b
    torch.cuda.empty_cache()
    # ---- single precision at 1024 x 768 x 70
    coeffs, b = system("latlon_1024x768x70")
    Href = MGHandle(*coeffs)
    xref, _ = Href.solve(b, tol=1e-12, raise_on_error=False)
    del Href
    b32 = b.float()
    single, mixed = {}, {}
    for name, code in methods.items():
        cap = args.krylov_maxit if name == "bicgstab_line" else 300
        H = MGHandle(*coeffs, method=code, mixed=1, maxit=cap)
        ms, (x32, info) = timed(lambda: H.solve_single(b32, tol=TOL, raise_on_error=False,
                                                        history_cap=cap + 64))
        hist = info["history"]
        err = float(torch.linalg.vector_norm(x32.double() - xref) / torch.linalg.vector_norm(xref))
        single[name] = {"ms": ms, "status": info["status"], "iterations": info["iterations"],
                        "best_rel_res": min(hist) if hist else None,
                        "best_at": hist.index(min(hist)) if hist else None,
                        "last_rel_res": hist[-1] if hist else None,
                        "error_vs_fp64_solution": err,
                        "history": [float("%.3e" % h) for h in hist[:60]]}
        Hm = MGHandle(*coeffs, method=code, mixed=1, maxit=100, inner_maxit=40)
        x = torch.zeros_like(b)
        Hm.solve_mixed(b, x, tol=TOL, raise_on_error=False)
        x.zero_()
        ms, (_, info) = timed(lambda: Hm.solve_mixed(b, x, tol=TOL, raise_on_error=False))
        mixed[name] = {"ms": ms, "status": info["status"], "refinement_steps": info["iterations"],
                       "fp32_iterations": info["inner_iterations"], "rel_res": info["rel_res"]}
        del H, Hm, x
        torch.cuda.empty_cache()
    out["latlon_1024x768x70_single"] = single
    out["latlon_1024x768x70_mixed"] = mixed
    print(json.dumps(out))


def run_ns(args):
    """The nonsymmetric comparison as its own JSON line (ns_measure)."""
    print(json.dumps(ns_measure(args.steps)))


def ns_measure(steps):
    """The nonsymmetric operator (the transport-augmented 1536 x 1152 x 70
    system, pe 0.3): FP64 BiCGStab preconditioned by the V-cycle to 1e-10 for
    H and for H^T (the adjoint solve of a differentiable nonsymmetric solve),
    the same with FP32 multigrid inside FP64 refinement, beside FP64
    BiCGStab on the symmetric operator without the transport, and the event
    times of the nonsymmetric fine-level kernels."""
    import torch

    from paper_2307_04528_gb300 import _lib as L
    from paper_2307_04528_gb300.solver import MGHandle, NSHandle

    w = WORKLOADS["latlon_1536x1152x70"]
    seed = workload_seed("latlon_1536x1152x70")
    P = make_ns_problem(w["nlon"], w["nlat"], w["nz"], w["sigma"], seed, pe=0.3)
    d = lambda a: torch.as_tensor(a, dtype=torch.float64).cuda()
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            out = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    b = d(P["b"])
    H = NSHandle(*(d(P[k]) for k in ("h", "tx", "ty", "tz", "txr", "tyr", "tzr")),
                 method=L.MG_METHOD_BICGSTAB, mixed=1)
    out = {"metric": "ms to 1e-10 rel residual, nonsymmetric 1536x1152x70 (transport pe 0.3), "
                     "FP64 BiCGStab + V-cycle: H and H^T (mixed_*: FP32 multigrid in FP64 "
                     "refinement)", "unit": "ms", "n_gpus": 1,
           "higher_is_better": False, "dtype": "f64", "data": "synthetic",
           "config": {"workload": "latlon_1536x1152x70_transport", "unknowns": int(b.numel()),
                      "tol": TOL, "levels": H.num_levels}}
    x = torch.zeros_like(b)
    for tr in (False, True):
        def solve():
            x.zero_()
            return H.solve(b, x, tol=TOL, transpose=tr, raise_on_error=False)
        ms, (_, info) = timed(solve, steps)
        out["transpose" if tr else "forward"] = {
            "ms": ms, "status": info["status"], "iterations": info["iterations"],
            "rel_res": info["rel_res"]}
    # FP32 multigrid (BiCGStab + V-cycle) inside FP64 refinement, H and H^T
    for tr in (False, True):
        def solve_mixed():
            x.zero_()
            return H.solve_mixed(b, x, tol=TOL, transpose=tr, raise_on_error=False)
        ms, (_, info) = timed(solve_mixed, steps)
        out["mixed_transpose" if tr else "mixed_forward"] = {
            "ms": ms, "status": info["status"], "refinement_steps": info["iterations"],
            "fp32_iterations": info["inner_iterations"], "rel_res": info["rel_res"]}
    out["value"] = out["forward"]["ms"]
    gen = torch.Generator(device="cuda").manual_seed(0)
    u = torch.randn(b.shape, generator=gen, device="cuda", dtype=torch.float64)
    n = b.numel()
    kern = []
    for name, fn, words in (("k_ns_stencil (H x)", lambda: H.apply(u), 9),
                            ("k_ns_stencil (H^T x, transposed stencil)",
                             lambda: H.apply(u, transpose=True), 9),
                            ("k_ns_smooth (sweep)", lambda: H.level_smooth(0, b, u), 10),
                            ("k_ns_smooth (from zero)", lambda: H.level_smooth(0, b, None), 5)):
        ms, _ = timed(fn, 10)
        kern.append({"kernel": name, "avg_ms": ms, "alg_bytes": 8.0 * words * n,
                     "gbs": 8.0 * words * n / (ms * 1e-3) / 1e9})
    out["kernels_fine_level"] = kern
    del H, x, u
    torch.cuda.empty_cache()
    S = make_problem(w["nlon"], w["nlat"], w["nz"], w["sigma"], seed)
    Hs = MGHandle(*(d(S[k]) for k in ("tx", "ty", "tz", "h")), method=L.MG_METHOD_BICGSTAB)
    bs = d(S["b"])
    xs = torch.zeros_like(bs)

    def solve_sym():
        xs.zero_()
        return Hs.solve(bs, xs, tol=TOL, raise_on_error=False)
    ms, (_, info) = timed(solve_sym, steps)
    out["symmetric_same_method"] = {"ms": ms, "status": info["status"],
                                    "iterations": info["iterations"]}
    out["steps"] = steps
    del Hs, bs, xs
    torch.cuda.empty_cache()
    return out


def main():
    args = parse()
    if args.kernel:
        run_kernel(args)
        return
    if args.workload == "krylov":
        run_krylov(args)
        return
    if args.workload == "ensemble":
        run_ensemble(args)
        return
    if args.workload == "ns":
        run_ns(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
