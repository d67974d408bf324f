"""The numerical experiments of Sec. 3 on the cube (0,3)^3 of 27 unit patches
with the manufactured field A_ana (non-homogeneous tangential Dirichlet data,
nu = 1), one JSON line per run:

    python -m paper_2501_04340_gb300.experiments --exp 1 [--degrees 1 2 3]
        [--spans 2 3 4 6 8] [--max-gb 120]
    python -m paper_2501_04340_gb300.experiments --exp 2 [--degrees 1 2 3]
        [--nsub 2 ... 12] [--spans 4] [--max-gb 120]

The mesh size is the one of the paper's figures, h = 1 / (n * 27^(1/3)) =
1 / (3 n) for n knot spans per patch and direction (the element width relative
to the cube's edge). Experiment 1 varies h and the degree p on three subdomains
(the two L-shaped columns and the slab of workloads.three_columns_partition);
experiment 2 varies the number of subdomains (consecutive patches in snake
order, each checked to be simply connected) at h = 1 / 12 (n = 4). Every run
reports the coarse size n_gp, the PCG iterations to the relative residual 1e-6
(FP64 factors, one pass), the Lanczos estimate of kappa(M_D^-1 F_DP) from the
PCG coefficients, and eps_B against B_ana. The dense local blocks grow like the
square of the subdomain's DOFs: a run whose blocks would take more than
--max-gb of device memory is reported as skipped instead of run.
"""
from __future__ import annotations

import argparse
import json
import time


def _dense_bytes(q) -> int:
    """Device bytes of the dense per-subdomain blocks: K_rr as assembled and its
    factor (n_r^2 each), S_rIrI and W (n_I^2 each)."""
    return 8 * (2 * int(q["sum_nr2"]) + 2 * int(q["sum_nI2"]))


def run_one(ieti, wl, torch, p: int, spans: int, nsub: int, tol: float, max_bytes: float, exp: int) -> dict:
    prob = wl.paper_cube(p, spans, nsub=nsub)
    rec = {"experiment": exp, "p": p, "h": 1.0 / (3 * spans), "spans": spans, "nsub": nsub}
    hctx = ieti.ieti_create_host(prob)
    try:
        q = ieti.ieti_query(hctx)
    finally:
        ieti.ieti_destroy(hctx)
    rec.update({"nedge": q["nedge"], "n_gauged": q["n_gauged"], "m_r": q["m_r"], "n_gp": q["n_gp"],
                "max_nr": q["max_nr"], "dense_gb": round(_dense_bytes(q) / 1e9, 3)})
    if _dense_bytes(q) > max_bytes:
        rec["skipped"] = "dense local blocks above the memory cap"
        return rec
    ctx = ieti.ieti_create(prob)
    try:
        a = torch.zeros((1, q["nedge"]), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ieti.ieti_assemble(ctx)
        ieti.ieti_factor(ctx, ieti.IETI_FP64)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        info = ieti.ieti_solve(ctx, a, tol=tol, maxit=2000, allow_no_convergence=True)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        _, err2 = ieti.ieti_eval_B(ctx, a, prob.npatch_total, ref_kind=ieti.IETI_BREF_TRIG, ref_amp=[1.0])
        rec.update({"iterations": info.iterations, "kappa": info.kappa, "relres": info.relres,
                    "converged": info.converged, "eps_B": float(err2.sum()) ** 0.5,
                    "setup_s": round(t1 - t0, 4), "solve_s": round(t2 - t1, 4)})
    finally:
        ieti.ieti_destroy(ctx)
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--exp", type=int, choices=[1, 2], required=True)
    ap.add_argument("--degrees", type=int, nargs="+", default=[1, 2, 3])
    ap.add_argument("--spans", type=int, nargs="+", default=None)
    ap.add_argument("--nsub", type=int, nargs="+", default=list(range(2, 13)))
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--max-gb", type=float, default=120.0)
    args = ap.parse_args()

    import torch

    from paper_2501_04340_gb300 import ieti, workloads as wl

    cap = args.max_gb * 1e9
    if args.exp == 1:
        spans = args.spans or [2, 3, 4, 6, 8]
        for p in args.degrees:
            for n in spans:
                print(json.dumps(run_one(ieti, wl, torch, p, n, 3, args.tol, cap, 1)), flush=True)
    else:
        spans = (args.spans or [4])[0]
        for p in args.degrees:
            for ns in args.nsub:
                print(json.dumps(run_one(ieti, wl, torch, p, spans, ns, args.tol, cap, 2)), flush=True)


if __name__ == "__main__":
    main()
