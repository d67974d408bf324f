"""GPU parity of the non-homogeneous tangential Dirichlet data (Sec. 2 boundary
condition with the manufactured field of Sec. 3, IETI_SOURCE_TRIG) against the
oracle: the lifted loads j - K a_D per subdomain (FP64 on both sides, different
summation order: 1e-12), the solved field including its boundary coefficients
(1e-8 in the 2-norm, both precisions, as for the homogeneous cases) and the
flux error eps_B against B_ana (1e-10)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import boundary as bd, discretise as dz, fetidp as fd, monolithic as mono, post, topology as tp
from paper_2501_04340_gb300 import workloads as wl


@pytest.fixture(scope="module")
def ieti():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_04340_gb300 import ieti as m
    return m


# (p, spans per patch, subdomains): the three columns of the paper's layout, an
# uneven snake partition, and a two-subdomain split
CASES = [(2, 2, 3), (3, 1, 5), (1, 3, 2)]
AMPS = [1.0, -0.5]


def _oracle(p, spans, nsub):
    prob = wl.paper_cube(p, spans, nsub=nsub, nrhs=2, amps=AMPS)
    mesh, Kp, jp = dz.assemble_all(prob)
    aD = bd.boundary_projection(prob, mesh, bd.manufactured_A)
    jl = bd.lift(Kp, jp, aD, AMPS)
    topo = tp.build_topology(prob, mesh)
    a, _ = mono.solve(mesh, topo, Kp, jl)
    a = a + aD[:, None] * np.asarray(AMPS)[None, :]
    sysd = fd.build_system(prob, (mesh, Kp, jl), topo)
    return prob, mesh, sysd, a


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("case", CASES)
def test_lifted_loads_equal_oracle(ieti, case):
    prob, mesh, sysd, _ = _oracle(*case)
    ctx = ieti.ieti_create(prob)
    try:
        ieti.ieti_assemble(ctx)
        for k, s in enumerate(sysd.subs):
            r_lib = np.concatenate([ieti.ieti_get_dofmap(ctx, 4, k), ieti.ieti_get_dofmap(ctx, 5, k)])
            pos = {int(e): i for i, e in enumerate(s.r_ids)}
            perm = np.array([pos[int(e)] for e in r_lib], dtype=np.int64)
            assert rel(ieti.ieti_get_block(ctx, 3, k), s.jr[perm]) < 1e-12
            if len(s.Cidx):
                assert rel(ieti.ieti_get_block(ctx, 4, k), s.jp) < 1e-12
    finally:
        ieti.ieti_destroy(ctx)


@pytest.mark.parametrize("case", CASES)
@pytest.mark.parametrize("prec", [0, 1])
def test_field_and_flux_error_equal_oracle(ieti, case, prec):
    prob, mesh, sysd, a_o = _oracle(*case)
    ctx = ieti.ieti_create(prob)
    try:
        ieti.ieti_assemble(ctx)
        ieti.ieti_factor(ctx, prec)
        a = torch.zeros((2, mesh.nedge), dtype=torch.float64, device="cuda")
        ieti.ieti_solve(ctx, a, tol=1e-11, maxit=400, tol_field=1e-12 if prec else 0.0)
        ah = a.cpu().numpy().T
        bnd = dz.dirichlet_edges(mesh)
        # the boundary coefficients are returned exactly as projected and scaled
        aD = ieti.ieti_get_boundary_data(ctx)
        for r, s in enumerate(AMPS):
            assert np.array_equal(ah[bnd, r], s * aD[bnd])
            assert np.linalg.norm(ah[:, r] - a_o[:, r]) <= 1e-8 * np.linalg.norm(a_o[:, r])
        # eps_B of the device field by the device and by the oracle's quadrature
        nB2, err2 = ieti.ieti_eval_B(ctx, a, prob.npatch_total, ref_kind=ieti.IETI_BREF_TRIG, ref_amp=AMPS)
        for r, s in enumerate(AMPS):
            _, eb = post.flux_l2(prob, mesh, ah, B_exact=lambda X: s * bd.manufactured_B(X), rhs=r)
            assert abs(np.sqrt(err2[r].sum()) - eb) <= 1e-10 * eb
    finally:
        ieti.ieti_destroy(ctx)


def test_flux_error_falls_like_h_to_the_p(ieti):
    """Sec. 3 on the cube (0,3)^3 with three slab subdomains: eps_B = O(h^p)."""
    for p, ns in ((1, (2, 4)), (2, (1, 2))):
        errs = []
        for n in ns:
            prob = wl.paper_cube(p, n)
            ctx = ieti.ieti_create(prob)
            try:
                ieti.ieti_assemble(ctx)
                ieti.ieti_factor(ctx, ieti.IETI_FP64)
                a = torch.zeros((1, dz.build_mesh(prob).nedge), dtype=torch.float64, device="cuda")
                ieti.ieti_solve(ctx, a, tol=1e-10)
                _, err2 = ieti.ieti_eval_B(ctx, a, prob.npatch_total, ref_kind=ieti.IETI_BREF_TRIG, ref_amp=[1.0])
                errs.append(np.sqrt(err2.sum()))
            finally:
                ieti.ieti_destroy(ctx)
        rate = np.log2(errs[0] / errs[1])
        assert rate > 0.8 * p, (p, errs)


def test_experiment_one_trends(ieti):
    """Experiment 1 of Sec. 3 at the coarse end of its range (h = 1/(3n) = 1/6
    and 1/12): the coarse size n_gp does not change with h and p, and
    kappa(M_D^-1 F_DP) and the PCG iterations at the paper's tolerance stay
    inside the ranges its figure plots."""
    import json
    import os
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_guides.json")))
    ngp = set()
    for p in (1, 2, 3):
        for n in (2, 4):
            prob = wl.paper_cube(p, n)
            ctx = ieti.ieti_create(prob)
            try:
                ngp.add(ieti.ieti_query(ctx)["n_gp"])
                ieti.ieti_assemble(ctx)
                ieti.ieti_factor(ctx, ieti.IETI_FP64)
                a = torch.zeros((1, dz.build_mesh(prob).nedge), dtype=torch.float64, device="cuda")
                info = ieti.ieti_solve(ctx, a, tol=g["pcg_tol"])
                lo, hi = g["exp1_axis_kappa"]
                assert lo <= info.kappa <= hi, (p, n, info.kappa)
                lo, hi = g["exp1_axis_iter"]
                assert lo <= info.iterations <= hi, (p, n, info.iterations)
            finally:
                ieti.ieti_destroy(ctx)
    assert len(ngp) == 1 and ngp.pop() > 0
