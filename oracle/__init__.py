"""Plain FP64 CPU oracle of the dual-primal IETI method for 3D magnetostatics.

TEST INFRASTRUCTURE ONLY. Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU baseline leg
(and its ``--impl reference`` arm) use it. It shares no code with the CUDA path;
the only common module is the seeded input generator
``paper_2501_04340_gb300.workloads``, which holds no method arithmetic.

Every function cites the passage of the paper (arXiv 2501.04340, "On Domain
Decomposition for Magnetostatic Problems in 3D") it follows. Readings of
passages where the paper is silent or ambiguous are marked "Reading:".

Modules
  splines     B-spline / edge-spline bases, Gauss rules            (Sec. 2, Eq. (3) space)
  discretise  glued multipatch mesh, Galerkin assembly of K_g, j_g (Eq. (3))
  topology    facets, wire basket, weights, Kruskal tree, DOF classes (Sec. 2.2, Fig. weights)
  fetidp      blocks, F, G, W, d, e, Dirichlet preconditioner, PCG,
              recovery (Eqs. (4)-(9))
  monolithic  gauged global direct solve (Eq. (3) with the same tree)
  post        B = curl a at quadrature points and the flux error (Sec. 3)

Parity status: every function is pinned by a ``-m "not gpu"`` test in
``tests/test_oracle_*.py``; none is "parity unpinned".
"""
