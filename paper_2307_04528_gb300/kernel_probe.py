"""Run one fine-level kernel of the multigrid a fixed number of times.

Used to time a kernel in isolation with CUDA events and to drive `ncu`
captures on a case small enough to profile (a few GB on the device) while
every array still exceeds the 129 MB L2.  Inputs come from the seeded
generator; the kernel is called through the library's per-level C ABI.

    python -m paper_2307_04528_gb300.kernel_probe --shape 512 384 70 \
        --kernel smooth32 --launches 5
"""
from __future__ import annotations

import argparse
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# kernel name -> (precision, per-level entry point, words per cell)
KERNELS = {
    "smooth32": (1, "smooth", 8),
    "smooth32_dot": (1, "smooth_dot", 8),
    "smooth32_zero": (1, "smooth0", 5),
    "resid32": (1, "residual", 7),
    "apply32": (1, "apply", 6),
    "restrict32": (1, "restrict", None),
    "resid_restrict32": (1, "resid_restrict", None),
    "presmooth_restrict32": (1, "presmooth_restrict", None),
    "prolong32": (1, "prolong", None),
    "smooth64": (0, "smooth", 8),
    "smooth64_zero": (0, "smooth0", 5),
    "resid64": (0, "residual", 7),
    "apply64": (0, "apply", 6),
}


def main():
    import torch

    from synthetic import make_problem
    from paper_2307_04528_gb300.solver import MGHandle

    ap = argparse.ArgumentParser()
    ap.add_argument("--shape", type=int, nargs=3, default=[512, 384, 70],
                    metavar=("NLON", "NLAT", "NZ"))
    ap.add_argument("--kernel", choices=sorted(KERNELS), default="smooth32")
    ap.add_argument("--launches", type=int, default=5)
    ap.add_argument("--sigma", type=float, default=0.2)
    args = ap.parse_args()
    nlon, nlat, nz = args.shape
    P = make_problem(nlon, nlat, nz, args.sigma, 3000)
    d = lambda a, dt=torch.float64: torch.as_tensor(a).to("cuda", dt)
    H = MGHandle(d(P["tx"]), d(P["ty"]), d(P["tz"]), d(P["h"]), mixed=1)
    prec, op, words = KERNELS[args.kernel]
    dt = torch.float32 if prec == 1 else torch.float64
    gen = torch.Generator(device="cuda").manual_seed(0)
    shape = (nz, nlat, nlon)
    b = torch.randn(shape, generator=gen, device="cuda", dtype=dt)
    u = torch.randn(shape, generator=gen, device="cuda", dtype=dt)
    cshape = H.level_shape(1) if H.num_levels > 1 else shape
    ec = torch.randn(cshape, generator=gen, device="cuda", dtype=dt)

    def run():
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
    if words:
        nbytes = words * (4 if prec == 1 else 8) * n
        out.update(alg_bytes=nbytes, gbs=nbytes / (ms * 1e-3) / 1e9)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
