"""Writes the stored oracle solutions under tests/golden/ (run once on a CPU;
calls only the oracle and the seeded input generator).

cube64_p3n8_sub16.npz -- the 64-patch cube in 16 subdomains (p = 3, 8 spans,
per-patch nu log-uniform in [1, 1e3], seed 2; the sine source): the FP64
dual-primal solve of Eqs. (7)-(9) with PCG to a relative residual of 1e-13,
  a_idx, a_val  the nonzero entries of the field a (every other entry is 0),
  nB            ||B||_L2 per patch of B = curl a (Sec. 3 error norm),
  relres_K      ||j - K a|| / ||j|| of the gauged global system (Eq. (3)),
  iters, kappa  PCG iterations and the Lanczos estimate of kappa(M^-1 F).

Usage: python tests/golden/make_golden.py [name ...]
"""
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import discretise as dz, fetidp as fd, monolithic as mono, post, topology as tp  # noqa: E402
from paper_2501_04340_gb300 import workloads as wl  # noqa: E402

CASES = {"cube64_p3n8_sub16": lambda: wl.cube64_p3n8_sub16()}


def make(name):
    t0 = time.time()
    prob = CASES[name]()
    mesh, Kp, jp = dz.assemble_all(prob)
    t1 = time.time()
    topo = tp.build_topology(prob, mesh)
    sysd = fd.build_system(prob, (mesh, Kp, jp), topo)
    t2 = time.time()
    sol = fd.solve(sysd, tol=1e-13, maxit=2000)
    t3 = time.time()
    K, j = mono.global_matrix(Kp, jp)
    keep = ~topo.dirichlet & ~topo.tree
    res = (j - K @ sol.a)[keep]
    relres = float(np.linalg.norm(res) / np.linalg.norm(j[keep]))
    nB = np.array([[post.flux_l2(prob, mesh, sol.a, rhs=r, patches=[q])[0] for q in range(prob.npatch_total)]
                   for r in range(prob.nrhs)])
    idx = np.flatnonzero(np.any(sol.a != 0, axis=1))
    out = os.path.join(HERE, name + ".npz")
    np.savez_compressed(out, a_idx=idx.astype(np.int32), a_val=sol.a[idx], nedge=mesh.nedge, nB=nB,
                        relres_K=relres, iters=np.array(sol.iters), kappa=np.array(sol.kappa),
                        relres=np.array(sol.relres))
    print(f"{name}: assembly {t1 - t0:.1f} s, blocks {t2 - t1:.1f} s, solve {t3 - t2:.1f} s, "
          f"iterations {sol.iters}, kappa {sol.kappa}, ||j - K a||/||j|| = {relres:.2e}, "
          f"jump {sol.jump:.2e}, {os.path.getsize(out) / 1e6:.2f} MB")


if __name__ == "__main__":
    for n in (sys.argv[1:] or list(CASES)):
        make(n)
