"""Pins of the oracle's Galerkin assembly (Eq. (3)) against closed forms."""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import discretise as dz, splines
from paper_2501_04340_gb300 import workloads as wl


def _one_box(p, spans, L, nu=1.0, source_kind=wl.SOURCE_SINE, params=None):
    prob = wl.unit_cube(p, (1, 1, 1), [[spans[0]], [spans[1]], [spans[2]]], nu=[nu],
                        source_kind=source_kind, source_params=params)
    prob.ctrl[..., 0] *= L[0]
    prob.ctrl[..., 1] *= L[1]
    prob.ctrl[..., 2] *= L[2]
    return prob


def _gram_1d(p, n, fa, fb):
    """int_0^1 f_a f_b for 1D families 'N', 'dN', 'D' built from scipy BSplines,
    with a 12-point Gauss rule per span (exact for these piecewise polynomials)."""
    t = splines.open_uniform_knots(p, n)
    nb = n + p

    def family(f):
        out = []
        if f == "N":
            for i in range(nb):
                out.append(BSpline(t, np.eye(nb)[i], p))
        elif f == "dN":
            for i in range(nb):
                out.append(BSpline(t, np.eye(nb)[i], p).derivative())
        else:  # Curry-Schoenberg D_i = p/(t_{i+p+1}-t_{i+1}) N_{i+1,p-1}
            m = len(t) - p
            for i in range(nb - 1):
                c = np.zeros(m); c[i + 1] = p / (t[i + p + 1] - t[i + 1])
                out.append(BSpline(t, c, p - 1))
        return out

    A, B = family(fa), family(fb)
    x, w = np.polynomial.legendre.leggauss(12)
    G = np.zeros((len(A), len(B)))
    for s in range(n):
        xs = (s + 0.5 * (x + 1)) / n
        ws = 0.5 * w / n
        va = np.array([f(xs) for f in A])
        vb = np.array([f(xs) for f in B])
        G += (va * ws) @ vb.T
    return G


# curl of the reference edge functions as (component, sign, (fx, fy, fz))
_CURL = {
    0: [(1, +1, ("D", "N", "dN")), (2, -1, ("D", "dN", "N"))],
    1: [(0, -1, ("N", "D", "dN")), (2, +1, ("dN", "D", "N"))],
    2: [(0, +1, ("N", "dN", "D")), (1, -1, ("dN", "N", "D"))],
}


@pytest.mark.parametrize("p,spans,L", [(1, (2, 3, 1), (1.0, 0.5, 2.0)),
                                       (2, (2, 2, 3), (0.3, 1.0, 0.7)),
                                       (3, (1, 2, 2), (1.0, 1.0, 1.0))])
def test_affine_patch_equals_kronecker_closed_form(p, spans, L):
    nu = 2.5
    prob = _one_box(p, spans, L, nu=nu)
    mesh, Kp, _ = dz.assemble_all(prob)
    K = Kp[0].toarray()
    det = L[0] * L[1] * L[2]
    g = [nu * L[c] ** 2 / det for c in range(3)]
    blocks = [[None] * 3 for _ in range(3)]
    for d in range(3):
        for e in range(3):
            acc = 0.0
            for (c1, s1, f1) in _CURL[d]:
                for (c2, s2, f2) in _CURL[e]:
                    if c1 != c2:
                        continue
                    G = [_gram_1d(p, spans[k], f1[k], f2[k]) for k in range(3)]
                    acc = acc + g[c1] * s1 * s2 * np.kron(G[2], np.kron(G[1], G[0]))
            blocks[d][e] = acc
    Kref = np.block(blocks)
    assert np.abs(K - Kref).max() < 1e-12 * np.abs(Kref).max()


def test_load_vector_for_constant_current():
    """J = (c0, c1, c2) constant on a box: j of an edge-d function is
    c_d * prod_{k != d} L_k * int D * prod int N (closed form, int D_i = 1)."""
    p, spans, L = 2, (2, 3, 2), (0.5, 1.0, 2.0)
    cst = np.array([1.5, -0.5, 2.0])
    prob = _one_box(p, spans, L, source_kind=wl.SOURCE_PATCHWISE, params=cst)
    mesh, _, jp = dz.assemble_all(prob)
    j = jp[0][:, 0]
    intN = []
    for d in range(3):
        t = splines.open_uniform_knots(p, spans[d])
        intN.append(np.array([(t[i + p + 1] - t[i]) / (p + 1) for i in range(spans[d] + p)]))
    ref = []
    for d in range(3):
        fac = [intN[k] if k != d else np.ones(spans[d] + p - 1) for k in range(3)]
        area = np.prod([L[k] for k in range(3) if k != d])
        ref.append(cst[d] * area * np.kron(fac[2], np.kron(fac[1], fac[0])))
    np.testing.assert_allclose(j, np.concatenate(ref), atol=1e-13)


def _curved(prob, amp=0.05, seed=0):
    """Smoothly perturb interior control points (non-affine, still regular map)."""
    rng = np.random.default_rng(seed)
    c = prob.ctrl.copy()
    N2, N1, N0, _ = c.shape
    for d in range(3):
        c[1:-1, 1:-1, 1:-1, d] += amp * rng.uniform(-1, 1, (N2 - 2, N1 - 2, N0 - 2)) / max(N0, N1, N2)
    c[1:-1, 1:-1, 1:-1, 3] = 1.0 + 0.2 * rng.uniform(0, 1, (N2 - 2, N1 - 2, N0 - 2))
    prob.ctrl = c
    return prob


@pytest.mark.parametrize("make", [lambda: wl.cube8_p2n4(spans=2),
                                  lambda: _curved(wl.unit_cube(3, (2, 1, 1), 2)),
                                  lambda: _curved(wl.unit_cube(2, (1, 2, 2), [[3], [2, 2], [1, 2]]), seed=3)])
def test_curl_of_gradients_vanishes(make):
    """K G_inc = 0: gradients of the H1 basis are the incidence columns and lie in
    the kernel of the curl-curl matrix, for affine and NURBS maps alike."""
    prob = make()
    mesh, Kp, _ = dz.assemble_all(prob)
    G = dz.incidence(mesh)
    for K in Kp:
        KG = K @ G
        assert abs(KG).max() < 1e-11 * abs(K).max()
        Kd = K.toarray()
        assert np.allclose(Kd, Kd.T, atol=1e-13 * abs(Kd).max())
        assert np.linalg.eigvalsh(Kd).min() > -1e-10 * abs(Kd).max()


def test_periodic_direction_mesh_counts():
    """A periodic direction has as many edges per line as control points."""
    prob = wl.unit_cube(2, (3, 1, 1), 2)
    prob.periodic0 = True
    mesh = dz.build_mesh(prob)
    assert mesh.N[0] == 3 * (2 + 2 - 1)
    assert mesh.edge_ext[0][0] == mesh.N[0]
    t, h = mesh.edge_endpoints()
    assert len(np.unique(np.stack([t, h], 1), axis=0)) == mesh.nedge
