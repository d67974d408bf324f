"""Glued multipatch control mesh and Galerkin assembly (oracle, test infrastructure).

Sec. 2: patches Omega_mp^(j) = F^(j)((0,1)^3) with fully shared patch-facets;
Eq. (3): (K_g)_ij = int nu curl w_j . curl w_i dV, (j_g)_i = int J . w_i dV.

Mesh conventions (data format shared with the CUDA path's host code, written
independently there):
  * node (i, j, k) of the glued control net has id i + N0 (j + N1 k);
  * an edge of direction d runs from node (i,j,k) (tail) to (i,j,k) + e_d (head),
    wrapping in direction 0 when it is periodic; its orientation is the
    direction of increasing parameter, inherited by every local copy;
  * edge ids: all direction-0 edges, then direction-1, then direction-2, each
    block lexicographic with i fastest over its own index extents.
Reading (Sec. 2.2: the gauge identifies DOFs with mesh edges): the edge DOF
(i,j,k) of direction d is the coefficient of the edge function whose 1D factor
in direction d is D_i and N in the other directions.
Reading (quadrature, not stated): p+1 Gauss-Legendre points per direction per
knot span.
Reading (Dirichlet, Sec. 2, n x A = 0): every edge lying in a boundary face of
the glued control net is removed.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Tuple

import numpy as np
import scipy.sparse as sp

from . import splines

SOURCE_SINE, SOURCE_FOURIER, SOURCE_PATCHWISE, SOURCE_TRIG = 0, 1, 2, 3


@dataclasses.dataclass
class Mesh:
    p: int
    N: Tuple[int, int, int]
    periodic0: bool
    npatch: Tuple[int, int, int]
    nspan: List[List[int]]
    starts: List[List[int]]          # per direction: first control index of each slab
    edge_ext: List[Tuple[int, int, int]]  # per direction: index extents of that edge block
    edge_off: List[int]
    nedge: int
    nnode: int

    def node_id(self, i, j, k):
        return i + self.N[0] * (j + self.N[1] * k)

    def edge_id(self, d, i, j, k):
        e = self.edge_ext[d]
        return self.edge_off[d] + i + e[0] * (j + e[1] * k)

    def edge_endpoints(self):
        """(tail, head) node ids of every edge, by edge id."""
        tails = np.empty(self.nedge, np.int64)
        heads = np.empty(self.nedge, np.int64)
        for d in range(3):
            e = self.edge_ext[d]
            k, j, i = np.meshgrid(np.arange(e[2]), np.arange(e[1]), np.arange(e[0]), indexing="ij")
            i, j, k = i.ravel(), j.ravel(), k.ravel()
            ids = self.edge_id(d, i, j, k)
            hi, hj, hk = i.copy(), j.copy(), k.copy()
            if d == 0:
                hi = hi + 1
                if self.periodic0:
                    hi = hi % self.N[0]
            elif d == 1:
                hj = hj + 1
            else:
                hk = hk + 1
            tails[ids] = self.node_id(i, j, k)
            heads[ids] = self.node_id(hi, hj, hk)
        return tails, heads

    def edge_ijk(self):
        """(direction, i, j, k) of every edge, by edge id."""
        out = np.empty((self.nedge, 4), np.int64)
        for d in range(3):
            e = self.edge_ext[d]
            k, j, i = np.meshgrid(np.arange(e[2]), np.arange(e[1]), np.arange(e[0]), indexing="ij")
            ids = self.edge_id(d, i.ravel(), j.ravel(), k.ravel())
            out[ids, 0] = d
            out[ids, 1] = i.ravel()
            out[ids, 2] = j.ravel()
            out[ids, 3] = k.ravel()
        return out


def build_mesh(prob) -> Mesh:
    p = prob.p
    N = prob.grid_shape()
    starts = []
    for d in range(3):
        s, acc = [], 0
        for n in prob.nspan[d]:
            s.append(acc)
            acc += n + p - 1
        starts.append(s)
    ext, off, tot = [], [], 0
    for d in range(3):
        e = list(N)
        if not (d == 0 and prob.periodic0):
            e[d] -= 1
        ext.append(tuple(e))
        off.append(tot)
        tot += e[0] * e[1] * e[2]
    return Mesh(p=p, N=N, periodic0=prob.periodic0, npatch=prob.npatch, nspan=prob.nspan,
                starts=starts, edge_ext=ext, edge_off=off, nedge=tot, nnode=N[0] * N[1] * N[2])


def dirichlet_edges(mesh: Mesh) -> np.ndarray:
    """Boolean mask: edge lies in a boundary face of the glued control net
    (n x A = g_D = 0, Sec. 2)."""
    eijk = mesh.edge_ijk()
    d = eijk[:, 0]
    mask = np.zeros(mesh.nedge, bool)
    for dd in range(3):
        if dd == 0 and mesh.periodic0:
            continue
        idx = eijk[:, 1 + dd]
        on = ((idx == 0) | (idx == mesh.N[dd] - 1)) & (d != dd)
        mask |= on
    return mask


def boundary_nodes(mesh: Mesh) -> np.ndarray:
    mask = np.zeros(mesh.nnode, bool)
    k, j, i = np.meshgrid(np.arange(mesh.N[2]), np.arange(mesh.N[1]), np.arange(mesh.N[0]), indexing="ij")
    ijk = (i.ravel(), j.ravel(), k.ravel())
    ids = mesh.node_id(*ijk)
    for dd in range(3):
        if dd == 0 and mesh.periodic0:
            continue
        mask[ids[(ijk[dd] == 0) | (ijk[dd] == mesh.N[dd] - 1)]] = True
    return mask


def incidence(mesh: Mesh) -> sp.csr_matrix:
    """Signed edge-node incidence G (nedge x nnode): +1 at the head, -1 at the tail.
    With N_i' = D_{i-1} - D_i, grad of the H1 function of a node is sum_e G[e, node] w_e."""
    t, h = mesh.edge_endpoints()
    rows = np.concatenate([np.arange(mesh.nedge), np.arange(mesh.nedge)])
    cols = np.concatenate([h, t])
    vals = np.concatenate([np.ones(mesh.nedge), -np.ones(mesh.nedge)])
    return sp.csr_matrix((vals, (rows, cols)), shape=(mesh.nedge, mesh.nnode))


def patch_index(prob, a, b, c):
    return a + prob.npatch[0] * (b + prob.npatch[1] * c)


def patch_abc(prob, q):
    P0, P1 = prob.npatch[0], prob.npatch[1]
    return q % P0, (q // P0) % P1, q // (P0 * P1)


def patch_edges(prob, mesh: Mesh, q) -> np.ndarray:
    """Global ids of all edges in the closure of patch q (per-patch local order:
    direction, then local (i, j, k) with i fastest)."""
    a = patch_abc(prob, q)
    p = prob.p
    n = [prob.nspan[d][a[d]] for d in range(3)]
    st = [mesh.starts[d][a[d]] for d in range(3)]
    out = []
    for d in range(3):
        ext = [n[e] + p - (1 if e == d else 0) for e in range(3)]
        k, j, i = np.meshgrid(np.arange(ext[2]), np.arange(ext[1]), np.arange(ext[0]), indexing="ij")
        gi = st[0] + i.ravel()
        if mesh.periodic0:
            gi = gi % mesh.N[0]
        out.append(mesh.edge_id(d, gi, st[1] + j.ravel(), st[2] + k.ravel()))
    return np.concatenate(out)


def patch_nodes(prob, mesh: Mesh, q) -> np.ndarray:
    a = patch_abc(prob, q)
    p = prob.p
    n = [prob.nspan[d][a[d]] + p for d in range(3)]
    st = [mesh.starts[d][a[d]] for d in range(3)]
    k, j, i = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    gi = st[0] + i.ravel()
    if mesh.periodic0:
        gi = gi % mesh.N[0]
    return mesh.node_id(gi, st[1] + j.ravel(), st[2] + k.ravel())


# ----------------------------------------------------------------------------
# element data
# ----------------------------------------------------------------------------

def _tables_1d(p, nspan, s, xq):
    """1D tables on span s: N (p+1 x nq), N' (p+1 x nq), D (p x nq), local
    function indices s..s+p (H1) and s..s+p-1 (edge)."""
    t = splines.open_uniform_knots(p, nspan)
    nq = len(xq)
    N = np.zeros((p + 1, nq))
    dN = np.zeros((p + 1, nq))
    D = np.zeros((p, nq))
    for q, x in enumerate(xq):
        xx = (s + x) / nspan
        Nall = splines.h1_values(t, p, xx)
        dNall = splines.h1_derivs(t, p, xx)
        Dall = splines.edge_values(t, p, xx)
        N[:, q] = Nall[s:s + p + 1]
        dN[:, q] = dNall[s:s + p + 1] * 1.0
        D[:, q] = Dall[s:s + p]
    return N, dN, D


def source_values(prob, X: np.ndarray, q_patch: int) -> np.ndarray:
    """J at physical points X (..., 3) for every load case: (..., 3, nrhs)."""
    nr = prob.nrhs
    out = np.zeros(X.shape[:-1] + (3, nr))
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    if prob.source_kind == SOURCE_SINE:
        base = 2 * np.pi ** 2 * np.stack([np.sin(np.pi * y) * np.sin(np.pi * z),
                                          np.sin(np.pi * x) * np.sin(np.pi * z),
                                          np.sin(np.pi * x) * np.sin(np.pi * y)], axis=-1)
        for r in range(nr):
            out[..., :, r] = prob.source_params[r] * base
    elif prob.source_kind == SOURCE_FOURIER:
        pos = 0
        P = prob.source_params
        for r in range(nr):
            nm = int(P[pos]); pos += 1
            acc = np.zeros(X.shape[:-1] + (3,))
            for m in range(nm):
                k = P[pos:pos + 3]; cr = P[pos + 3:pos + 6]; ci = P[pos + 6:pos + 9]; pos += 9
                th = 2 * np.pi * (k[0] * x + k[1] * y + k[2] * z)
                acc += np.cos(th)[..., None] * cr - np.sin(th)[..., None] * ci
            out[..., :, r] = acc
    elif prob.source_kind == SOURCE_PATCHWISE:
        P = prob.source_params.reshape(nr, prob.npatch_total, 3)
        for r in range(nr):
            out[..., :, r] = P[r, q_patch]
    elif prob.source_kind == SOURCE_TRIG:
        # Sec. 3: curl curl A_ana = 3 A_ana (A_ana is divergence free and each
        # component is an eigenfunction of -Laplace with eigenvalue 3)
        base = 3.0 * np.stack([np.cos(y) * np.cos(z) * np.sin(x),
                               -2.0 * np.cos(x) * np.cos(z) * np.sin(y),
                               np.cos(x) * np.cos(y) * np.sin(z)], axis=-1)
        for r in range(nr):
            out[..., :, r] = prob.source_params[r] * base
    else:
        raise ValueError("unknown source kind")
    return out


def element_funcs(p, tabs):
    """Reference edge functions and their reference curls on one element.

    tabs = [(N, dN, D) per direction]. Returns (val, curl), each (nfunc, nq3, 3),
    functions ordered by component d, then local (a, b, c) with a fastest, and
    the local index triples (d, a, b, c) relative to the element's first function."""
    (N0, dN0, D0), (N1, dN1, D1), (N2, dN2, D2) = tabs
    nq = N0.shape[1]
    vals, curls, idx = [], [], []

    def tp(A, B, C):  # tensor product over (c, b, a) x (qz, qy, qx) -> (nf, nq3)
        T = np.einsum("ax,by,cz->cbazyx", A, B, C)
        return T.reshape(A.shape[0] * B.shape[0] * C.shape[0], nq ** 3)

    # direction 0: D(x) N(y) N(z) e_x; curl = (0, D N N', -D N' N)
    f = tp(D0, N1, N2)
    c1 = tp(D0, N1, dN2)
    c2 = -tp(D0, dN1, N2)
    z = np.zeros_like(f)
    vals.append(np.stack([f, z, z], -1)); curls.append(np.stack([z, c1, c2], -1))
    # direction 1: N(x) D(y) N(z) e_y; curl = (-N D N', 0, N' D N)
    f = tp(N0, D1, N2)
    c0 = -tp(N0, D1, dN2)
    c2 = tp(dN0, D1, N2)
    z = np.zeros_like(f)
    vals.append(np.stack([z, f, z], -1)); curls.append(np.stack([c0, z, c2], -1))
    # direction 2: N(x) N(y) D(z) e_z; curl = (N N' D, -N' N D, 0)
    f = tp(N0, N1, D2)
    c0 = tp(N0, dN1, D2)
    c1 = -tp(dN0, N1, D2)
    z = np.zeros_like(f)
    vals.append(np.stack([z, z, f], -1)); curls.append(np.stack([c0, c1, z], -1))
    for d in range(3):
        ext = [p + 1, p + 1, p + 1]
        ext[d] = p
        for c in range(ext[2]):
            for b in range(ext[1]):
                for a in range(ext[0]):
                    idx.append((d, a, b, c))
    return np.concatenate(vals, 0), np.concatenate(curls, 0), np.array(idx)


def _geometry(p, ctrl_loc, tabs_geo):
    """NURBS map on one element: physical points X (nq3, 3) and Jacobians DF (nq3, 3, 3)
    with DF[:, r, c] = d x_r / d xi_c, from the element's (p+1)^3 control points
    ctrl_loc (p+1, p+1, p+1, 4) indexed [c, b, a]."""
    (N0, dN0), (N1, dN1), (N2, dN2) = tabs_geo
    w = ctrl_loc[..., 3]
    P = ctrl_loc[..., :3]
    W = np.einsum("cba,ax,by,cz->zyx", w, N0, N1, N2)
    Wd = [np.einsum("cba,ax,by,cz->zyx", w, dN0, N1, N2),
          np.einsum("cba,ax,by,cz->zyx", w, N0, dN1, N2),
          np.einsum("cba,ax,by,cz->zyx", w, N0, N1, dN2)]
    wP = w[..., None] * P
    S = np.einsum("cbar,ax,by,cz->zyxr", wP, N0, N1, N2)
    Sd = [np.einsum("cbar,ax,by,cz->zyxr", wP, dN0, N1, N2),
          np.einsum("cbar,ax,by,cz->zyxr", wP, N0, dN1, N2),
          np.einsum("cbar,ax,by,cz->zyxr", wP, N0, N1, dN2)]
    X = S / W[..., None]
    DF = np.stack([(Sd[c] - X * Wd[c][..., None]) / W[..., None] for c in range(3)], -1)
    nq3 = X.shape[0] * X.shape[1] * X.shape[2]
    return X.reshape(nq3, 3), DF.reshape(nq3, 3, 3)


def _patch_element_loop(prob, mesh, q, nq=None):
    """Yield per element: (global edge ids of its functions, val, curl, X, DF, weights)."""
    p = prob.p
    a3 = patch_abc(prob, q)
    n = [prob.nspan[d][a3[d]] for d in range(3)]
    st = [mesh.starts[d][a3[d]] for d in range(3)]
    if nq is None:
        nq = p + 1
    xq, wq = splines.gauss_legendre(nq)
    cache = [{} for _ in range(3)]
    for d in range(3):
        for s in range(n[d]):
            cache[d][s] = _tables_1d(p, n[d], s, xq)
    W3 = np.einsum("z,y,x->zyx", wq, wq, wq).ravel()
    for s2 in range(n[2]):
        for s1 in range(n[1]):
            for s0 in range(n[0]):
                s = (s0, s1, s2)
                tabs = [cache[d][s[d]] for d in range(3)]
                val, curl, idx = element_funcs(p, tabs)
                # geometry: control points of the element, scaled to physical span size
                gi = st[0] + s0 + np.arange(p + 1)
                if mesh.periodic0:
                    gi = gi % mesh.N[0]
                gj = st[1] + s1 + np.arange(p + 1)
                gk = st[2] + s2 + np.arange(p + 1)
                ctrl_loc = prob.ctrl[np.ix_(gk, gj, gi)]
                # all tables are functions of the patch parameter xi in (0,1)^3:
                # N' = dN/dxi and D_i use the patch knot vector, so DF = dx/dxi
                tg = [(tabs[d][0], tabs[d][1]) for d in range(3)]
                X, DF = _geometry(p, ctrl_loc, tg)
                # global edge ids of the element functions
                gids = np.empty(len(idx), np.int64)
                for f, (d, aa, bb, cc) in enumerate(idx):
                    ii = st[0] + s0 + aa
                    if mesh.periodic0:
                        ii = ii % mesh.N[0]
                    gids[f] = mesh.edge_id(d, ii, st[1] + s1 + bb, st[2] + s2 + cc)
                # weights in patch parameter space: element measure 1/(n0 n1 n2)
                wts = W3 / (n[0] * n[1] * n[2])
                yield gids, val, curl, X, DF, wts


def assemble_patch(prob, mesh, q, nq=None):
    """Patch contribution to K_g and j_g (Eq. (3)) as COO triplets and a dense
    load block: returns (rows, cols, vals, gid_rhs, rhs_vals). ``nq`` Gauss
    points per direction per span (default p+1, the reading used throughout)."""
    nu = prob.nu[q]
    R, C, V = [], [], []
    jr_ids, jr_vals = [], []
    for gids, val, curl, X, DF, wts in _patch_element_loop(prob, mesh, q, nq=nq):
        det = np.linalg.det(DF)
        # dV = |det DF| dxi (a patch map may reverse orientation);
        # curl w = DF curl_hat / det ; int nu curl_i . curl_j = sum_q w nu c_i^T DF^T DF c_j / |det|
        M = np.einsum("qra,qrb->qab", DF, DF) * (nu * wts / np.abs(det))[:, None, None]
        Y = np.einsum("qab,jqb->jqa", M, curl)
        nf = curl.shape[0]
        E = curl.reshape(nf, -1) @ Y.reshape(nf, -1).T
        # j_i = int J . DF^{-T} w_hat |det| = sum_q w |det| (DF^{-1} J) . w_hat
        J = source_values(prob, X, q)                       # (nq3, 3, nrhs)
        DFinv = np.linalg.inv(DF)
        G = np.einsum("qab,qbr->qar", DFinv, J) * (wts * np.abs(det))[:, None, None]
        je = val.reshape(val.shape[0], -1) @ G.reshape(-1, G.shape[-1])
        R.append(np.repeat(gids, len(gids)))
        C.append(np.tile(gids, len(gids)))
        V.append(E.ravel())
        jr_ids.append(gids)
        jr_vals.append(je)
    return (np.concatenate(R), np.concatenate(C), np.concatenate(V),
            np.concatenate(jr_ids), np.concatenate(jr_vals, 0))


def assemble_all(prob, mesh=None, nq=None):
    """Per-patch matrices K_patch (global edge indexing, CSR) and loads j_patch
    (dense nedge x nrhs). Subdomain matrices K^(k) (Sec. 2, block-diagonal K) and
    the global K_g are sums of these."""
    if mesh is None:
        mesh = build_mesh(prob)
    Kp, jp = [], []
    for q in range(prob.npatch_total):
        r, c, v, ji, jv = assemble_patch(prob, mesh, q, nq=nq)
        Kp.append(sp.csr_matrix((v, (r, c)), shape=(mesh.nedge, mesh.nedge)))
        jj = np.zeros((mesh.nedge, prob.nrhs))
        np.add.at(jj, ji, jv)
        jp.append(jj)
    return mesh, Kp, jp
