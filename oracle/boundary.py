"""Non-homogeneous tangential Dirichlet data (oracle, test infrastructure).

Sec. 2 states the boundary condition n x A = g_D; Sec. 3 prescribes the data of
the manufactured field A_ana on the cube (0,3)^3 with nu = 1, whose source is
J = curl curl A_ana = 3 A_ana (A_ana is divergence free and -Laplace A_ana =
3 A_ana).

Reading (the paper does not say how the boundary coefficients of the discrete
field are chosen): the coefficients of the edges lying in the Dirichlet faces
(the DOFs removed for g_D = 0) are the L2 projection of the tangential trace of
g_D onto the tangential traces of the edge functions, over the whole boundary
at once, since the faces share the coefficients of the edges on the box's
edges. The other coefficients solve Eq. (3) with the lifted loads
j - K a_D; the discrete field is their sum.

Only axis-aligned affine box patches (the cube of Sec. 3): on a face normal to
axis n, an edge function of direction d != n has the single tangential
component D_i(xi_d) N_j(xi_e) / L_d (covariant map with DF = diag(L); the
factor in direction n is 1 on the face for the boundary index, 0 otherwise).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import discretise as dz
from . import splines


def manufactured_A(X):
    """A_ana of Sec. 3 at points X (..., 3)."""
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    return np.stack([np.cos(y) * np.cos(z) * np.sin(x),
                     -2.0 * np.cos(x) * np.cos(z) * np.sin(y),
                     np.cos(x) * np.cos(y) * np.sin(z)], -1)


def manufactured_B(X):
    """B_ana = curl A_ana of Sec. 3 at points X (..., 3)."""
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    return np.stack([-3.0 * np.cos(x) * np.sin(y) * np.sin(z),
                     np.zeros_like(x),
                     3.0 * np.cos(z) * np.sin(x) * np.sin(y)], -1)


def _patch_box(prob, mesh, q):
    """Lower corner and edge lengths of the affine box patch q."""
    a3 = dz.patch_abc(prob, q)
    st = [mesh.starts[d][a3[d]] for d in range(3)]
    n = [prob.nspan[d][a3[d]] for d in range(3)]
    lo = prob.ctrl[st[2], st[1], st[0], :3]
    hi = prob.ctrl[st[2] + n[2] + prob.p - 1, st[1] + n[1] + prob.p - 1, st[0] + n[0] + prob.p - 1, :3]
    return lo, hi - lo, st, n, a3


def boundary_projection(prob, mesh, g, nq=None):
    """Coefficients a_D (nedge,) of the edges in the Dirichlet faces: the L2
    projection of the tangential trace of g (a function of points (..., 3)
    returning (..., 3)) over the boundary; zero on every other edge."""
    if prob.periodic0:
        raise ValueError("boundary projection: periodic directions are not supported")
    p = prob.p
    if nq is None:
        nq = p + 1
    xq, wq = splines.gauss_legendre(nq)
    rows, cols, vals = [], [], []
    rhs = np.zeros(mesh.nedge)
    for q in range(prob.npatch_total):
        lo, L, st, n, a3 = _patch_box(prob, mesh, q)
        for ax in range(3):
            for side in (0, 1):
                if a3[ax] != (0 if side == 0 else prob.npatch[ax] - 1):
                    continue
                cidx = 0 if side == 0 else mesh.N[ax] - 1      # control index along the normal
                xn = lo[ax] + (0.0 if side == 0 else L[ax])
                tang = [c for c in range(3) if c != ax]
                for d in tang:                                 # component / edge direction
                    e = tang[0] if tang[1] == d else tang[1]
                    td = splines.open_uniform_knots(p, n[d])
                    te = splines.open_uniform_knots(p, n[e])
                    for sd in range(n[d]):
                        for se in range(n[e]):
                            xd = (sd + xq) / n[d]
                            xe = (se + xq) / n[e]
                            # D_i(xi_d) (p functions of the span), N_j(xi_e) (p + 1)
                            Dd = np.array([splines.edge_values(td, p, t)[sd:sd + p] for t in xd]).T
                            Ne = np.array([splines.h1_values(te, p, t)[se:se + p + 1] for t in xe]).T
                            # physical points of the face quadrature
                            X = np.zeros((nq, nq, 3))
                            X[..., ax] = xn
                            X[..., d] = (lo[d] + L[d] * xd)[:, None]
                            X[..., e] = (lo[e] + L[e] * xe)[None, :]
                            gd = g(X)[..., d]                                  # (nq_d, nq_e)
                            w2 = np.outer(wq, wq) * (L[d] / n[d]) * (L[e] / n[e])
                            # traces (i, j, qd, qe) = D_i N_j / L_d
                            T = np.einsum("iq,jr->ijqr", Dd, Ne) / L[d]
                            ids = np.empty((p, p + 1), np.int64)
                            for i in range(p):
                                for j in range(p + 1):
                                    c = [0, 0, 0]
                                    c[ax] = cidx
                                    c[d] = st[d] + sd + i
                                    c[e] = st[e] + se + j
                                    ids[i, j] = mesh.edge_id(d, c[0], c[1], c[2])
                            Tf = T.reshape(p * (p + 1), -1)
                            Wf = w2.ravel()
                            Me = (Tf * Wf) @ Tf.T
                            fe = Tf @ (Wf * gd.ravel())
                            idf = ids.ravel()
                            rows.append(np.repeat(idf, len(idf)))
                            cols.append(np.tile(idf, len(idf)))
                            vals.append(Me.ravel())
                            np.add.at(rhs, idf, fe)
    M = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(mesh.nedge, mesh.nedge))
    bnd = dz.dirichlet_edges(mesh)
    idx = np.flatnonzero(bnd)
    aD = np.zeros(mesh.nedge)
    aD[idx] = spla.spsolve(M[idx][:, idx].tocsc(), rhs[idx])
    return aD


def lift(Kpatch, jpatch, aD, amps):
    """Patch loads with the lifting, j_q - K_q a_D amp_r per load case r
    (Eq. (3) for the coefficients off the Dirichlet faces)."""
    out = []
    for Kq, jq in zip(Kpatch, jpatch):
        ka = Kq @ aD
        out.append(jq - ka[:, None] * np.asarray(amps)[None, :])
    return out
