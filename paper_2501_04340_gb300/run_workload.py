"""Solve one synthetic workload end to end and print the solve report as JSON.

    python -m paper_2501_04340_gb300.run_workload [--patches 4] [--spans 8]
        [--degree 3] [--block 2 2 1] [--precision fp32|fp64] [--tol 1e-8]
        [--tol-field 1e-8] [--repeat 1] [--named NAME]

The default is the 64-patch unit cube with 16 subdomains of 2x2x1 patches and
per-patch reluctivity log-uniform in [1, 1e3] (seed 2). --spans and --patches
give smaller or larger variants of the same layout (for instance to profile a
case that holds a few GB on the device). --named runs one of the named
workloads instead: cube512_p3_uneven64 (512 patches, 64 uneven subdomains, 32
Fourier load cases), machine_annulus (NURBS annulus, 16 load cases) or
cube64_uneven8 (its reduced uneven variant, 32 load cases); the report then
adds the per-phase times.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--patches", type=int, default=4, help="patches per direction")
    ap.add_argument("--spans", type=int, default=8)
    ap.add_argument("--degree", type=int, default=3)
    ap.add_argument("--block", type=int, nargs=3, default=[2, 2, 1], help="patches per subdomain")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--tol-field", type=float, default=1e-8)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--named", default=None, choices=["cube512_p3_uneven64", "machine_annulus", "cube64_uneven8"])
    args = ap.parse_args()

    import torch

    from paper_2501_04340_gb300 import ieti, workloads as wl

    if args.named:
        prob = getattr(wl, args.named)()
    else:
        P = args.patches
        rng = np.random.default_rng(2)
        nu = 10.0 ** rng.uniform(0.0, 3.0, size=P ** 3)
        sub = wl.block_partition((P, P, P), tuple(args.block))
        prob = wl.unit_cube(args.degree, (P, P, P), args.spans, sub_of_patch=sub, nu=nu,
                            name=f"cube{P ** 3}_p{args.degree}n{args.spans}")
    prec = ieti.IETI_FP32_IR if args.precision == "fp32" else ieti.IETI_FP64
    ctx = ieti.ieti_create(prob)
    try:
        q = ieti.ieti_query(ctx)
        a = torch.zeros((prob.nrhs, q["nedge"]), dtype=torch.float64, device="cuda")
        phases = {}
        for _ in range(args.repeat):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ieti.ieti_assemble(ctx)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            ieti.ieti_factor(ctx, prec)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            info = ieti.ieti_solve(ctx, a, tol=args.tol, maxit=2000,
                                   tol_field=args.tol_field if prec == ieti.IETI_FP32_IR else 0.0)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            phases = {"assemble_s": round(t1 - t0, 4), "factor_s": round(t2 - t1, 4),
                      "solve_s": round(wall - (t2 - t0), 4)}
        print(json.dumps({"workload": prob.name, "precision": args.precision, "wall_s": round(wall, 4),
                          "pcg_iterations": info.iterations, "refinement_steps": info.refinement_steps,
                          "relres": info.relres, "field_residual": info.global_relres,
                          "kappa": info.kappa, "converged": info.converged, "nedge": q["nedge"],
                          "m_r": q["m_r"], "n_gp": q["n_gp"], "nrhs": prob.nrhs, "nsub": prob.nsub,
                          "device_bytes": q["bytes_device"], "fp64_fallback": info.fp64_fallback,
                          "launches": ieti.ieti_launch_count(ctx), **phases}))
    finally:
        ieti.ieti_destroy(ctx)


if __name__ == "__main__":
    main()
