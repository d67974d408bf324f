"""Pins of the oracle's rational patch maps and of its Fourier loads.

Sec. 2: patches are images of (0,1)^3 under spline/NURBS maps F^(j); Eq. (3)
integrates nu curl w_j . curl w_i and J . w_i over the mapped patches with the
covariant Piola push-forward. These tests fix the oracle against facts that do
not come from the oracle itself:
  * an exact quarter-annulus (rational arcs degree-elevated to p = 3) must give
    the closed-form map x = r(xi_1) (cos theta(xi_0), sin theta(xi_0)) + z e_z,
    its Jacobian and its volume pi (r2^2 - r1^2) L / 4;
  * the curl-curl matrix and the loads are invariant under a rigid rotation of
    the control net (with the source rotated along), which fails for a
    transposed Jacobian in the Piola maps;
  * the Fourier-source loads on a box equal separable 1D integrals of the
    B-spline factors against exp(2 pi i k.x), computed with scipy's adaptive
    quadrature.
"""
import math

import numpy as np
import pytest
from scipy import integrate
from scipy.interpolate import BSpline

from oracle import discretise as dz, splines
from paper_2501_04340_gb300 import workloads as wl


def _annulus_sector(p=3, patches=(2, 2, 1), spans=((2, 3), (2, 2), (2,)), r1=0.05, r2=0.1, L=0.1,
                    arc=math.pi / 2):
    return wl.annulus(p, patches, [list(s) for s in spans], r1, r2, L, arc=arc)


def _closed_form(prob, q, s, xi, r1, r2, L, arc):
    """Map and Jacobian of the exact shell sector at patch-local parameters xi (n x 3)."""
    a, b, c = dz.patch_abc(prob, q)
    P0, P1, P2 = prob.npatch
    dth = arc / P0
    rb = np.linspace(r1, r2, P1 + 1)
    zb = np.linspace(0.0, L, P2 + 1)
    u = 2 * xi[:, 0] - 1
    T = math.tan(dth / 4)
    th = a * dth + dth / 2 + 2 * np.arctan(T * u)
    dth_dxi = 4 * T / (1 + (T * u) ** 2)
    r = rb[b] + (rb[b + 1] - rb[b]) * xi[:, 1]
    z = zb[c] + (zb[c + 1] - zb[c]) * xi[:, 2]
    X = np.stack([r * np.cos(th), r * np.sin(th), z], -1)
    DF = np.zeros((len(xi), 3, 3))
    DF[:, 0, 0] = -r * np.sin(th) * dth_dxi
    DF[:, 1, 0] = r * np.cos(th) * dth_dxi
    DF[:, 0, 1] = (rb[b + 1] - rb[b]) * np.cos(th)
    DF[:, 1, 1] = (rb[b + 1] - rb[b]) * np.sin(th)
    DF[:, 2, 2] = zb[c + 1] - zb[c]
    return X, DF


def _element_xi(prob, q, nq):
    """Patch-local parameters of the Gauss points of every element of patch q,
    in the order of the oracle's element loop (x fastest inside an element)."""
    a3 = dz.patch_abc(prob, q)
    n = [prob.nspan[d][a3[d]] for d in range(3)]
    xq, _ = splines.gauss_legendre(nq)
    out = []
    for s2 in range(n[2]):
        for s1 in range(n[1]):
            for s0 in range(n[0]):
                zz, yy, xx = np.meshgrid(xq, xq, xq, indexing="ij")
                out.append(np.stack([(s0 + xx.ravel()) / n[0], (s1 + yy.ravel()) / n[1],
                                     (s2 + zz.ravel()) / n[2]], -1))
    return out


@pytest.mark.parametrize("nq", [4, 6])
def test_rational_map_is_the_exact_quarter_annulus(nq):
    r1, r2, L, arc = 0.05, 0.1, 0.1, math.pi / 2
    prob = _annulus_sector(r1=r1, r2=r2, L=L, arc=arc)
    mesh = dz.build_mesh(prob)
    for q in range(prob.npatch_total):
        xis = _element_xi(prob, q, nq)
        for xi, (gids, val, curl, X, DF, wts) in zip(xis, dz._patch_element_loop(prob, mesh, q, nq=nq)):
            Xe, DFe = _closed_form(prob, q, None, xi, r1, r2, L, arc)
            assert np.abs(X - Xe).max() <= 1e-12 * r2
            assert np.abs(DF - DFe).max() <= 1e-12 * np.abs(DFe).max()
            # the mapped points lie on the exact circles
            assert np.abs(np.hypot(X[:, 0], X[:, 1]) - np.hypot(Xe[:, 0], Xe[:, 1])).max() <= 1e-13


def test_quarter_annulus_volume():
    r1, r2, L = 0.05, 0.1, 0.1
    prob = _annulus_sector(r1=r1, r2=r2, L=L)
    mesh = dz.build_mesh(prob)
    vol = 0.0
    for q in range(prob.npatch_total):
        for gids, val, curl, X, DF, wts in dz._patch_element_loop(prob, mesh, q, nq=10):
            vol += np.sum(wts * np.abs(np.linalg.det(DF)))
    exact = math.pi * (r2 ** 2 - r1 ** 2) * L / 4
    assert abs(vol - exact) <= 1e-12 * exact


def _rotation(axis, angle):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    Kx = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(angle) * Kx + (1 - math.cos(angle)) * Kx @ Kx


def _rotated(prob, R, J=None):
    ctrl = prob.ctrl.copy()
    ctrl[..., :3] = prob.ctrl[..., :3] @ R.T
    out = wl.Problem(**{**prob.__dict__, "ctrl": ctrl})
    if J is not None:
        out.source_params = (J @ R.T).ravel()
    return out


@pytest.mark.parametrize("kind", ["box", "sector"])
def test_stiffness_and_loads_are_rotation_invariant(kind):
    rng = np.random.default_rng(11)
    if kind == "box":
        prob = wl.unit_cube(2, (1, 1, 1), [[2], [3], [1]], source_kind=wl.SOURCE_PATCHWISE,
                            source_params=np.zeros(3))
        prob.ctrl[..., 0] *= 0.7
        prob.ctrl[..., 2] *= 1.3
        R = _rotation([1.0, 2.0, -0.5], 0.8)
    else:
        prob = _annulus_sector(p=3, patches=(1, 1, 1), spans=((3,), (2,), (2,)))
        prob.source_kind = wl.SOURCE_PATCHWISE
        R = _rotation([0.0, 0.0, 1.0], 1.1)
    J = rng.standard_normal((1, 1, 3))
    prob.source_params = J.ravel()
    mesh, K0, j0 = dz.assemble_all(prob)
    _, K1, j1 = dz.assemble_all(_rotated(prob, R, J))
    K0, K1 = K0[0].toarray(), K1[0].toarray()
    assert np.abs(K1 - K0).max() <= 1e-12 * np.abs(K0).max()
    assert np.abs(j1[0] - j0[0]).max() <= 1e-12 * np.abs(j0[0]).max()
    # a transposed Jacobian in the curl map would break the invariance
    assert not np.allclose(R @ R.T @ np.diag([1, 2, 3]), R @ np.diag([1, 2, 3]) @ R.T)


def _basis(p, n, fam):
    t = splines.open_uniform_knots(p, n)
    nb = n + p
    if fam == "N":
        return t, [BSpline(t, np.eye(nb)[i], p) for i in range(nb)]
    m = len(t) - p
    out = []
    for i in range(nb - 1):   # Curry-Schoenberg D_i = p / (t_{i+p+1} - t_{i+1}) N_{i+1,p-1}
        c = np.zeros(m)
        c[i + 1] = p / (t[i + p + 1] - t[i + 1])
        out.append(BSpline(t, c, p - 1))
    return t, out


def _fourier_1d(p, n, fam, kappa):
    """int_0^1 f_i(xi) exp(i kappa xi) dxi for every function of the family, by
    adaptive quadrature span by span (real and imaginary parts)."""
    t, fs = _basis(p, n, fam)
    out = np.zeros(len(fs), complex)
    for i, f in enumerate(fs):
        for s in range(n):
            a, b = s / n, (s + 1) / n
            re = integrate.quad(lambda x: f(x) * math.cos(kappa * x), a, b, epsabs=1e-14, epsrel=1e-12)[0]
            im = integrate.quad(lambda x: f(x) * math.sin(kappa * x), a, b, epsabs=1e-14, epsrel=1e-12)[0]
            out[i] += re + 1j * im
    return out


def test_fourier_loads_equal_separable_integrals():
    p, spans, Ls = 3, (2, 1, 2), (0.8, 1.0, 0.6)
    modes = [((1.0, 0.0, -1.0), (0.3, -1.2, 0.7), (0.5, 0.2, -0.4)),
             ((0.0, 2.0, 1.0), (-0.8, 0.1, 0.9), (1.1, -0.6, 0.3))]
    params = [float(len(modes))]
    for k, cr, ci in modes:
        params += list(k) + list(cr) + list(ci)
    prob = wl.unit_cube(p, (1, 1, 1), [[spans[0]], [spans[1]], [spans[2]]], source_kind=wl.SOURCE_FOURIER,
                        source_params=np.array(params))
    for d in range(3):
        prob.ctrl[..., d] *= Ls[d]
    mesh, _, jp = dz.assemble_all(prob, nq=14)
    j = jp[0][:, 0]
    vol = Ls[0] * Ls[1] * Ls[2]
    ref = np.zeros(mesh.nedge)
    for k, cr, ci in modes:
        c = np.array(cr) + 1j * np.array(ci)
        I = {}
        for e in range(3):
            kap = 2 * math.pi * k[e] * Ls[e]
            I[e, "N"] = _fourier_1d(p, spans[e], "N", kap)
            I[e, "D"] = _fourier_1d(p, spans[e], "D", kap)
        for d in range(3):
            f = ["D" if e == d else "N" for e in range(3)]
            T = np.einsum("k,j,i->kji", I[2, f[2]], I[1, f[1]], I[0, f[0]])
            nk, nj, ni = T.shape
            kk, jj, ii = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
            ids = mesh.edge_id(d, ii.ravel(), jj.ravel(), kk.ravel())
            ref[ids] += (vol / Ls[d]) * np.real(c[d] * T.ravel())
    assert np.abs(j - ref).max() <= 1e-12 * np.abs(ref).max()
