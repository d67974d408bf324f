"""Pins of the oracle's dual-primal method (Eqs. (4)-(10)) against the
monolithic gauged solve and the mathematics of the method."""
import json
import os

import numpy as np
import pytest

from oracle import discretise as dz, topology as tp, fetidp as fd, monolithic as mono, post
from paper_2501_04340_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_guides.json")

CASES = [lambda: wl.cube8_p2n4(),
         lambda: wl.small_cases()[1],
         lambda: wl.small_cases()[2],
         lambda: wl.small_cases()[3],
         lambda: wl.unit_cube(2, (4, 4, 2), 1, sub_of_patch=wl.block_partition((4, 4, 2), (2, 2, 1)),
                              nu=10.0 ** np.random.default_rng(1).uniform(0, 3, 32), nrhs=2,
                              source_params=[1.0, -0.5])]


@pytest.mark.parametrize("make", CASES)
def test_dual_primal_equals_monolithic(make):
    """The dual-primal solution (Eqs. (7)-(9)) is the gauged monolithic solution."""
    prob = make()
    mesh, Kp, jp = dz.assemble_all(prob)
    topo = tp.build_topology(prob, mesh)
    a_m, _ = mono.solve(mesh, topo, Kp, jp)
    sysd = fd.build_system(prob, (mesh, Kp, jp), topo)
    sol = fd.solve(sysd, tol=1e-12)
    assert np.linalg.norm(sol.a - a_m) <= 1e-9 * np.linalg.norm(a_m)
    assert sol.jump < 1e-10          # multiplier jumps B a vanish at convergence


def test_interface_operator_spd_and_symmetric():
    sysd = fd.build_system(wl.cube8_p2n4(spans=2))
    op = fd.InterfaceOperator(sysd)
    A = op.dense()
    assert np.abs(A - A.T).max() < 1e-12 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0
    # the paper's coarse matrix F is negative definite
    assert np.linalg.eigvalsh(op.F).max() < 0


def test_schur_complement_is_inverse_of_inverse_block():
    """S_rIrI = K_II - K_IV K_VV^-1 K_VI equals ((K_rr^-1)_II)^-1 (block inverse identity)."""
    sysd = fd.build_system(wl.small_cases()[3])
    for s in sysd.subs:
        nI = len(s.Brow)
        E = np.zeros((s.Krr.shape[0], nI)); E[s.nV:] = np.eye(nI)
        Z = s.lu.solve(E)[s.nV:]
        S = s.KII - s.KIV @ s.KVV_lu.solve(s.KIV.T) if s.nV else s.KII
        assert np.abs(np.linalg.inv(Z) - S).max() < 1e-8 * np.abs(S).max()


def test_flux_is_gauge_invariant():
    """Two different spanning trees give different a but the same B = curl a."""
    prob = wl.small_cases()[3]
    mesh, Kp, jp = dz.assemble_all(prob)
    t1 = tp.build_topology(prob, mesh)
    t2 = tp.build_topology(prob, mesh, reverse_ties=True)
    assert np.any(t1.tree != t2.tree)
    s1 = fd.solve(fd.build_system(prob, (mesh, Kp, jp), t1), tol=1e-12)
    s2 = fd.solve(fd.build_system(prob, (mesh, Kp, jp), t2), tol=1e-12)
    assert np.linalg.norm(s1.a - s2.a) > 1e-3 * np.linalg.norm(s1.a)
    n1, _ = post.flux_l2(prob, mesh, s1.a)
    _, d12 = post.flux_l2(prob, mesh, s1.a, B_exact=None)
    # B difference: curl of (a1 - a2) must vanish
    nd, _ = post.flux_l2(prob, mesh, s1.a - s2.a)
    assert nd < 1e-9 * n1


@pytest.mark.parametrize("p,ns", [(1, [2, 4, 8]), (2, [1, 2, 4])])
def test_flux_error_rate_is_h_to_the_p(p, ns):
    """eps_B = O(h^p) for the manufactured field (Sec. 3, Fig. exp1 error panel)."""
    errs = []
    for n in ns:
        prob = wl.unit_cube(p, (2, 2, 2), n)
        mesh, Kp, jp = dz.assemble_all(prob)
        sysd = fd.build_system(prob, (mesh, Kp, jp))
        sol = fd.solve(sysd, tol=1e-10)
        _, e = post.flux_l2(prob, mesh, sol.a, post.sine_B, nq=p + 3)
        errs.append(e)
    rates = [np.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert abs(rates[-1] - p) < 0.35, rates


def test_condition_and_iterations_within_paper_bands():
    """kappa(M^-1 F_DP) and N_iter at tol 1e-6 inside the ranges plotted in
    Fig. exp1 (loose: the paper's layout is a different cube)."""
    g = json.load(open(GOLDEN))
    sysd = fd.build_system(wl.cube8_p2n4())
    sol = fd.solve(sysd, tol=g["pcg_tol"])
    lo, hi = g["exp1_axis_kappa"]
    assert lo <= sol.kappa[0] <= hi
    lo, hi = g["exp1_axis_iter"]
    assert lo <= sol.iters[0] <= hi


def test_preconditioner_only_changes_iterations():
    """Identity preconditioner vs Dirichlet preconditioner: same lambda; the
    Dirichlet one needs fewer iterations."""
    sysd = fd.build_system(wl.small_cases()[3])
    op = fd.InterfaceOperator(sysd)
    b = op.rhs()[:, 0]
    x1, it1, _, _ = fd.pcg(op, b, lambda r: r, tol=1e-12, maxit=2000)
    x2, it2, _, _ = fd.pcg(op, b, lambda r: fd.dirichlet_precond(sysd, r), tol=1e-12)
    assert np.linalg.norm(x1 - x2) < 1e-8 * np.linalg.norm(x1)
    assert it2 < it1
