"""Pins of the oracle's non-homogeneous tangential Dirichlet data (Sec. 2 boundary
condition, Sec. 3 manufactured field): the manufactured field against finite
differences, the boundary L2 projection against discrete gradients that it must
reproduce exactly, and the flux error of the lifted solve against the O(h^p)
rate of Sec. 3."""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import boundary as bd, discretise as dz, monolithic as mono, post, topology as tp
from paper_2501_04340_gb300 import workloads as wl


def _curl_fd(f, X, h=1e-4):
    """Central-difference curl of f at the points X (n, 3)."""
    J = np.zeros(X.shape[:-1] + (3, 3))      # J[..., r, c] = d f_r / d x_c
    for c in range(3):
        e = np.zeros(3); e[c] = h
        J[..., :, c] = (f(X + e) - f(X - e)) / (2 * h)
    return np.stack([J[..., 2, 1] - J[..., 1, 2], J[..., 0, 2] - J[..., 2, 0], J[..., 1, 0] - J[..., 0, 1]], -1)


def test_manufactured_field_and_source_by_finite_differences():
    """B_ana = curl A_ana, and the source of SOURCE_TRIG equals curl curl of the
    amplitude times A_ana (nu = 1)."""
    X = np.random.default_rng(0).uniform(0.0, 3.0, (40, 3))
    assert np.abs(_curl_fd(bd.manufactured_A, X) - bd.manufactured_B(X)).max() < 1e-7
    cc = _curl_fd(lambda Y: _curl_fd(bd.manufactured_A, Y, 1e-3), X, 1e-3)
    prob = wl.paper_cube(1, 1, nrhs=2, amps=[1.0, -0.5])
    J = dz.source_values(prob, X, 0)
    assert np.abs(J[..., 0] - cc).max() < 1e-4
    assert np.abs(J[..., 1] + 0.5 * cc).max() < 1e-4
    # A_ana does not satisfy n x A = 0 on the cube's boundary
    Y = np.array([[0.0, 1.0, 1.3], [3.0, 0.4, 2.0]])
    assert np.abs(bd.manufactured_A(Y)[:, 1:]).max() > 0.1


def _glued_knots(p, spans, breaks):
    """Knot vector of the glued 1D space in physical coordinates: p-fold knots at
    the patch breaks (C^0 gluing), p+1 at the ends."""
    t = [breaks[0]] * (p + 1)
    for a, n in enumerate(spans):
        t += list(np.linspace(breaks[a], breaks[a + 1], n + 1)[1:-1])
        t += [breaks[a + 1]] * (p if a + 1 < len(spans) else p + 1)
    return np.array(t)


def _poly_coefficients(p, t, f):
    """Spline coefficients of the polynomial f (degree <= p) by collocation at
    the Greville abscissae (scipy's B-splines)."""
    n = len(t) - p - 1
    g = np.array([t[i + 1:i + p + 1].mean() for i in range(n)])
    A = BSpline.design_matrix(np.clip(g, t[0], t[-1] - 1e-14), t, p).toarray()
    A[-1] = 0.0
    A[-1, -1] = 1.0
    return np.linalg.solve(A, f(g))


@pytest.mark.parametrize("p", [1, 2, 3])
def test_projection_reproduces_traces_of_discrete_gradients(p):
    """For phi a tensor polynomial of degree <= p per direction, grad phi is a
    discrete field whose coefficients are the differences of phi's spline
    coefficients along each edge; the boundary L2 projection of its tangential
    trace returns exactly those coefficients on the Dirichlet edges."""
    spans = [[2, 1], [1], [1, 2]]
    Ls = (1.5, 0.7, 2.2)
    breaks = [np.linspace(0.0, Ls[0], 3), np.array([0.0, Ls[1]]), np.linspace(0.0, Ls[2], 3)]
    prob = wl.unit_cube(p, (2, 1, 2), spans)
    prob.ctrl[...] = wl.box_control_net(p, spans, breaks)
    mesh = dz.build_mesh(prob)
    fs = [lambda x: 0.3 + x ** p - 0.7 * x, lambda y: 1.0 - 0.4 * y ** p + y, lambda z: 0.2 * z ** p + 0.5]
    dfs = [lambda x: p * x ** (p - 1) - 0.7, lambda y: -0.4 * p * y ** (p - 1) + 1.0, lambda z: 0.2 * p * z ** (p - 1)]
    cs = [_poly_coefficients(p, _glued_knots(p, spans[d], breaks[d]), fs[d]) for d in range(3)]
    C = np.einsum("i,j,k->kji", cs[0], cs[1], cs[2])            # [k, j, i]

    def grad_phi(X):
        x, y, z = X[..., 0], X[..., 1], X[..., 2]
        return np.stack([dfs[0](x) * fs[1](y) * fs[2](z),
                         fs[0](x) * dfs[1](y) * fs[2](z),
                         fs[0](x) * fs[1](y) * dfs[2](z)], -1)

    aD = bd.boundary_projection(prob, mesh, grad_phi)
    expect = np.zeros(mesh.nedge)
    for d in range(3):
        e = mesh.edge_ext[d]
        k, j, i = np.meshgrid(np.arange(e[2]), np.arange(e[1]), np.arange(e[0]), indexing="ij")
        hk, hj, hi = k + (d == 2), j + (d == 1), i + (d == 0)
        expect[mesh.edge_id(d, i.ravel(), j.ravel(), k.ravel())] = (C[hk, hj, hi] - C[k, j, i]).ravel()
    bnd = dz.dirichlet_edges(mesh)
    assert np.abs(aD[~bnd]).max() == 0.0
    assert np.abs(aD[bnd] - expect[bnd]).max() < 1e-11 * np.abs(expect).max()


def _lifted_flux_error(p, spans):
    prob = wl.paper_cube(p, spans, nrhs=1, amps=[1.0])
    mesh, Kp, jp = dz.assemble_all(prob)
    aD = bd.boundary_projection(prob, mesh, bd.manufactured_A)
    jl = bd.lift(Kp, jp, aD, [1.0])
    topo = tp.build_topology(prob, mesh)
    a, _ = mono.solve(mesh, topo, Kp, jl)
    a = a + aD[:, None]
    _, e = post.flux_l2(prob, mesh, a, bd.manufactured_B, nq=p + 3)
    _, e0 = post.flux_l2(prob, mesh, a - aD[:, None], bd.manufactured_B, nq=p + 3)
    return e, e0


@pytest.mark.parametrize("p,ns", [(1, [1, 2]), (2, [1, 2])])
def test_flux_error_of_the_lifted_solve_falls_like_h_to_the_p(p, ns):
    """eps_B = O(h^p) on the cube (0,3)^3 of Sec. 3 with the boundary data of
    A_ana; without the boundary coefficients the error does not fall."""
    errs, errs0 = [], []
    for n in ns:
        e, e0 = _lifted_flux_error(p, n)
        errs.append(e)
        errs0.append(e0)
    rate = np.log2(errs[0] / errs[1])
    assert rate > 0.8 * p, (errs, rate)
    assert errs0[1] > 0.5 * errs0[0]
    assert errs[1] < 0.5 * errs0[1]
