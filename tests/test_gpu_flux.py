"""GPU flux density B = curl a and its L2 norms (Sec. 3 error eps_B) against the
oracle's quadrature, on boxes and on the curved, periodic NURBS ring.

Both sides use p+1 Gauss points per direction per span, so the per-patch
squared norms agree to rounding: 1e-12 relative to the largest patch value.
B at the Gauss points is compared with B = DF curl_hat(a) / det DF built from
the oracle's element data, also at 1e-12.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import discretise as dz, fetidp as fd, post, topology as tp
from paper_2501_04340_gb300 import workloads as wl


@pytest.fixture(scope="module")
def ieti():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_04340_gb300 import ieti as m
    return m


CASES = {
    "cube8_p2n4": lambda: wl.cube8_p2n4(),
    "ragged_p3": lambda: wl.unit_cube(3, (2, 2, 1), [[2, 3], [3, 2], [3]],
                                      sub_of_patch=np.array([0, 1, 0, 2], np.int32), nrhs=2,
                                      source_params=[1.0, -2.0]),
    "ring24_p3n2": lambda: wl.machine_annulus(n_ang=12, n_ax=1, spans=2, nrhs=2),
}


def _oracle_B(prob, mesh, a, rhs):
    """B at the Gauss points of every element, patch by patch, from the oracle's element data."""
    out = []
    for q in range(prob.npatch_total):
        for gids, val, curl, X, DF, wts in dz._patch_element_loop(prob, mesh, q):
            ch = np.einsum("iqa,i->qa", curl, a[gids, rhs])
            out.append(np.einsum("qra,qa->qr", DF, ch) / np.linalg.det(DF)[:, None])
    return np.concatenate(out)


@pytest.mark.parametrize("name", list(CASES))
def test_flux_norms_and_values_equal_oracle(ieti, name):
    prob = CASES[name]()
    mesh = dz.build_mesh(prob)
    rng = np.random.default_rng(3)
    nr = 2
    a = rng.standard_normal((mesh.nedge, nr))      # every edge, Dirichlet and tree edges included
    ctx = ieti.ieti_create(prob)
    try:
        nelem = sum(prob.nspan[0][q % prob.npatch[0]] * prob.nspan[1][(q // prob.npatch[0]) % prob.npatch[1]] *
                    prob.nspan[2][q // (prob.npatch[0] * prob.npatch[1])] for q in range(prob.npatch_total))
        nq3 = (prob.p + 1) ** 3
        a_d = torch.tensor(a.T.copy(), dtype=torch.float64, device="cuda")
        Bq = torch.zeros((nr, nelem * nq3 * 3), dtype=torch.float64, device="cuda")
        nB2, err2 = ieti.ieti_eval_B(ctx, a_d, prob.npatch_total, B=Bq)
        assert err2 is None
        Bh = Bq.cpu().numpy()
        for r in range(nr):
            ref = np.array([post.flux_l2(prob, mesh, a, rhs=r, patches=[q])[0] ** 2
                            for q in range(prob.npatch_total)])
            assert np.abs(nB2[r] - ref).max() <= 1e-12 * ref.max()
            Bo = _oracle_B(prob, mesh, a, r)
            assert np.abs(Bh[r].reshape(-1, 3) - Bo).max() <= 1e-12 * np.abs(Bo).max()
    finally:
        ieti.ieti_destroy(ctx)


def test_flux_error_of_the_manufactured_solution(ieti):
    """eps_B of Sec. 3 for the sine source with nu = 1 (exact B known): the
    device value equals the oracle's on the same field, and it falls with the
    mesh size at the rate of Sec. 3 (O(h^p))."""
    errs = []
    for spans in (2, 4):
        prob = wl.cube8_p2n4(spans=spans)
        mesh, Kp, jp = dz.assemble_all(prob)
        ctx = ieti.ieti_create(prob)
        try:
            ieti.ieti_assemble(ctx)
            ieti.ieti_factor(ctx, ieti.IETI_FP64)
            a = torch.zeros((1, mesh.nedge), dtype=torch.float64, device="cuda")
            ieti.ieti_solve(ctx, a, tol=1e-12, tol_field=1e-13)
            nB2, err2 = ieti.ieti_eval_B(ctx, a, prob.npatch_total, ref_kind=ieti.IETI_BREF_SINE, ref_amp=[1.0])
            ah = a.cpu().numpy().T
            nb, eb = post.flux_l2(prob, mesh, ah, B_exact=post.sine_B)
            assert abs(np.sqrt(nB2.sum()) - nb) <= 1e-12 * nb
            assert abs(np.sqrt(err2.sum()) - eb) <= 1e-10 * eb
            errs.append(np.sqrt(err2.sum()))
        finally:
            ieti.ieti_destroy(ctx)
    rate = np.log2(errs[0] / errs[1])
    assert 1.7 <= rate <= 2.6, rate      # p = 2: second order in h


def test_eval_B_rejects_bad_arguments(ieti):
    prob = wl.cube8_p2n4(spans=1)
    ctx = ieti.ieti_create(prob)
    try:
        a = torch.zeros((1, dz.build_mesh(prob).nedge), dtype=torch.float64, device="cuda")
        with pytest.raises(ieti.IetiError, match="INVALID_ARG"):
            ieti.ieti_eval_B(ctx, a, prob.npatch_total, nrhs=65)
        with pytest.raises(ieti.IetiError, match="INVALID_ARG"):
            ieti.ieti_eval_B(ctx, a, prob.npatch_total, ref_kind=7, ref_amp=[1.0])
    finally:
        ieti.ieti_destroy(ctx)
