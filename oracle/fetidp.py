"""Dual-primal tearing and interconnecting, step by step (oracle, test
infrastructure).

Sec. 2.1: block-diagonal K = diag(K^(k)) (Eq. (4) context), dual-primal split
a = (a_r, a_p), a_p = C_p p (Eq. (5)), local elimination (Eq. (6)), interface
problem, coarse problem and local recovery (Eqs. (7)-(9)) with
  F = C^T K_pr K_rr^-1 K_rp C - C^T K_pp C,   G = B_r K_rr^-1 K_rp C,
  W = B_r K_rr^-1 B_r^T,  d = C^T K_pr K_rr^-1 j_r - C^T j_p,  e = B_r K_rr^-1 j_r,
PCG on the interface problem with the Dirichlet preconditioner of Eq. (10).

The interface problem S lam = G F^-1 d - e (Eq. (7)) is solved in the equivalent
SPD form  F_DP lam = b  with  F_DP = -S = W - G F^-1 G^T  and  b = e - G F^-1 d.
Readings:
  * D_s (Eq. (10)): rho-scaling after Klawonn-Widlund, per subdomain: the row of
    the multiplier coupling k and l is weighted in k's block by nu_l/(nu_k+nu_l)
    (nu at that edge: max over the subdomain's patches containing it). For a
    homogeneous nu this is the multiplicity scaling 1/2, which for CG is the same
    as the paper's D_s = I.
  * PCG stops when ||b - F_DP lam_k||_2 <= tol ||b||_2 (recursively updated residual).
"""
from __future__ import annotations

import dataclasses
from typing import List

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import discretise as dz
from . import topology as tp


@dataclasses.dataclass
class Subdomain:
    r_ids: np.ndarray       # global edge ids of r dofs, order [V, I]
    nV: int
    P_ids: np.ndarray
    Krr: sp.csc_matrix
    Krp: np.ndarray
    Kpp: np.ndarray
    jr: np.ndarray          # (n_r, nrhs)
    jp: np.ndarray          # (n_p, nrhs)
    lu: object              # factorisation of K_rr
    Brow: np.ndarray        # dual index of each I dof
    Bsign: np.ndarray
    Cidx: np.ndarray        # global primal index of each P dof
    Dscale: np.ndarray      # rho-scaling weight of each I dof
    KVV_lu: object
    KII: np.ndarray
    KIV: np.ndarray


@dataclasses.dataclass
class DPSystem:
    prob: object
    mesh: object
    topo: object
    subs: List[Subdomain]
    m_r: int
    n_gp: int
    Kpatch: list
    jpatch: list


def subdomain_matrix(prob, Kpatch, jpatch, k):
    """K^(k) and j^(k): sums over the patches of subdomain k (Sec. 2.1)."""
    K = None
    j = None
    for q in range(prob.npatch_total):
        if prob.sub_of_patch[q] != k:
            continue
        K = Kpatch[q] if K is None else K + Kpatch[q]
        j = jpatch[q] if j is None else j + jpatch[q]
    return K.tocsr(), j


def build_system(prob, assembled=None, topo=None) -> DPSystem:
    if assembled is None:
        assembled = dz.assemble_all(prob)
    mesh, Kpatch, jpatch = assembled
    if topo is None:
        topo = tp.build_topology(prob, mesh)
    subs = []
    for k in range(topo.nsub):
        K, j = subdomain_matrix(prob, Kpatch, jpatch, k)
        r_ids = np.concatenate([topo.V[k], topo.I[k]])
        Pk = topo.P[k]
        Krr = K[r_ids][:, r_ids].tocsc()
        Krp = K[r_ids][:, Pk].toarray()
        Kpp = K[Pk][:, Pk].toarray()
        lu = spla.splu(Krr)
        nV = len(topo.V[k])
        KVV = K[topo.V[k]][:, topo.V[k]].tocsc()
        KVV_lu = spla.splu(KVV) if nV > 0 else None
        KII = K[topo.I[k]][:, topo.I[k]].toarray()
        KIV = K[topo.I[k]][:, topo.V[k]].toarray()
        # rho-scaling weights (reading of D_s in Eq. (10))
        Dsc = np.empty(len(topo.I[k]))
        for t, (e, nuk) in enumerate(zip(topo.I[k], topo.nu_edge[k])):
            nul = None
            for l in range(topo.nsub):
                if l == k:
                    continue
                pos = np.searchsorted(topo.I[l], e)
                if pos < len(topo.I[l]) and topo.I[l][pos] == e:
                    nul = topo.nu_edge[l][pos]
                    break
            Dsc[t] = nul / (nuk + nul)
        subs.append(Subdomain(r_ids=r_ids, nV=nV, P_ids=Pk, Krr=Krr, Krp=Krp, Kpp=Kpp,
                              jr=j[r_ids], jp=j[Pk], lu=lu, Brow=topo.dual_of_I[k],
                              Bsign=topo.sign_of_I[k], Cidx=topo.primal_of_P[k], Dscale=Dsc,
                              KVV_lu=KVV_lu, KII=KII, KIV=KIV))
    return DPSystem(prob=prob, mesh=mesh, topo=topo, subs=subs, m_r=len(topo.dual_edges),
                    n_gp=len(topo.primal_edges), Kpatch=Kpatch, jpatch=jpatch)


# ----------------------------------------------------------------------------
# operators of Eqs. (7)-(9)
# ----------------------------------------------------------------------------

def _BrT(s: Subdomain, lam):
    """B_r^(k)T lam: local r-vector (zero on V, signed multipliers on I)."""
    u = np.zeros((s.Krr.shape[0],) + lam.shape[1:])
    u[s.nV:] = s.Bsign.reshape((-1,) + (1,) * (lam.ndim - 1)) * lam[s.Brow]
    return u


def _Br_add(s: Subdomain, v, out):
    """out += B_r^(k) v."""
    np.add.at(out, s.Brow, s.Bsign.reshape((-1,) + (1,) * (v.ndim - 1)) * v[s.nV:])


def _Ct_add(s: Subdomain, x, out):
    np.add.at(out, s.Cidx, x)


def coarse_matrix(sys: DPSystem):
    """The paper's F = C^T K_pr K_rr^-1 K_rp C - C^T K_pp C (negative definite)."""
    F = np.zeros((sys.n_gp, sys.n_gp))
    for s in sys.subs:
        if len(s.Cidx) == 0:
            continue
        X = s.lu.solve(s.Krp)
        loc = s.Krp.T @ X - s.Kpp
        F[np.ix_(s.Cidx, s.Cidx)] += loc
    return F


def G_matrix(sys: DPSystem):
    """G = B_r K_rr^-1 K_rp C (m_r x n_gp)."""
    G = np.zeros((sys.m_r, sys.n_gp))
    for s in sys.subs:
        if len(s.Cidx) == 0:
            continue
        X = s.lu.solve(s.Krp)               # n_r x n_p
        tmp = np.zeros((sys.m_r, len(s.Cidx)))
        _Br_add(s, X, tmp)
        for c, gc in enumerate(s.Cidx):
            G[:, gc] += tmp[:, c]
    return G


def apply_W(sys: DPSystem, lam):
    """W lam = B_r K_rr^-1 B_r^T lam."""
    y = np.zeros_like(lam)
    for s in sys.subs:
        _Br_add(s, s.lu.solve(_BrT(s, lam)), y)
    return y


def dense_W(sys: DPSystem):
    return apply_W(sys, np.eye(sys.m_r))


def vectors_d_e(sys: DPSystem):
    """d = C^T K_pr K_rr^-1 j_r - C^T j_p and e = B_r K_rr^-1 j_r."""
    nr = sys.prob.nrhs
    d = np.zeros((sys.n_gp, nr))
    e = np.zeros((sys.m_r, nr))
    for s in sys.subs:
        v = s.lu.solve(s.jr)
        _Br_add(s, v, e)
        if len(s.Cidx):
            _Ct_add(s, s.Krp.T @ v - s.jp, d)
    return d, e


class InterfaceOperator:
    """F_DP = W - G F^-1 G^T (the negated interface matrix S of Eq. (7))."""

    def __init__(self, sys: DPSystem):
        self.sys = sys
        self.F = coarse_matrix(sys)
        self.G = G_matrix(sys)
        self.Finv_G_T = np.linalg.solve(self.F, self.G.T) if sys.n_gp else np.zeros((0, sys.m_r))

    def __call__(self, lam):
        y = apply_W(self.sys, lam)
        if self.sys.n_gp:
            y = y - self.G @ (self.Finv_G_T @ lam)
        return y

    def rhs(self):
        d, e = vectors_d_e(self.sys)
        self.d = d
        if self.sys.n_gp:
            return e - self.G @ np.linalg.solve(self.F, d)
        return e

    def dense(self):
        return self(np.eye(self.sys.m_r))


def dirichlet_precond(sys: DPSystem, r):
    """M_D^-1 r = sum_k D^(k) B_rI^(k) S_rIrI^(k) B_rI^(k)T D^(k) r  with
    S_rIrI = K_II - K_IV K_VV^-1 K_VI (Eq. (10), rho-scaling reading for D)."""
    z = np.zeros_like(r)
    for s in sys.subs:
        shape = (-1,) + (1,) * (r.ndim - 1)
        u = (s.Bsign * s.Dscale).reshape(shape) * r[s.Brow]
        t = s.KII @ u
        if s.nV > 0:
            t = t - s.KIV @ s.KVV_lu.solve(s.KIV.T @ u)
        np.add.at(z, s.Brow, (s.Bsign * s.Dscale).reshape(shape) * t)
    return z


def pcg(A, b, M, tol=1e-8, maxit=500, x0=None):
    """Textbook preconditioned CG (Sec. 2.1, 'typically PCG'), one right-hand side.
    Returns x, iterations, relative residual history, (alphas, betas)."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A(x)
    nb = np.linalg.norm(b)
    hist = [np.linalg.norm(r) / nb]
    alphas, betas = [], []
    if hist[-1] <= tol:
        return x, 0, hist, (alphas, betas)
    z = M(r)
    p = z.copy()
    rz = r @ z
    it = 0
    for it in range(1, maxit + 1):
        q = A(p)
        alpha = rz / (p @ q)
        x = x + alpha * p
        r = r - alpha * q
        alphas.append(alpha)
        hist.append(np.linalg.norm(r) / nb)
        if hist[-1] <= tol:
            break
        z = M(r)
        rz_new = r @ z
        beta = rz_new / rz
        betas.append(beta)
        p = z + beta * p
        rz = rz_new
    return x, it, hist, (alphas, betas)


def lanczos_condition(alphas, betas):
    """kappa(M^-1 F_DP) estimate from the CG coefficients (tridiagonal Lanczos
    matrix T: T_jj = 1/a_j + b_{j-1}/a_{j-1}, T_{j,j+1} = sqrt(b_j)/a_j)."""
    n = len(alphas)
    if n == 0:
        return 1.0
    T = np.zeros((n, n))
    for j in range(n):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < n and j < len(betas):
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    ev = np.linalg.eigvalsh(T)
    return ev[-1] / ev[0]


@dataclasses.dataclass
class DPSolution:
    lam: np.ndarray          # (m_r, nrhs)
    p: np.ndarray            # (n_gp, nrhs)
    a_r: List[np.ndarray]    # per subdomain (n_rk, nrhs)
    a: np.ndarray            # global (nedge, nrhs)
    iters: List[int]
    relres: List[float]
    kappa: List[float]
    jump: float              # ||B_r a_r|| / ||a||


def solve(sys: DPSystem, tol=1e-8, maxit=500, lam0=None) -> DPSolution:
    """Eqs. (7)-(9): PCG on the interface problem, then the coarse and local
    recovery."""
    op = InterfaceOperator(sys)
    b = op.rhs()
    nr = sys.prob.nrhs
    lam = np.zeros((sys.m_r, nr))
    its, rel, kap = [], [], []
    for c in range(nr):
        x0 = None if lam0 is None else lam0[:, c]
        x, it, hist, (al, be) = pcg(op, b[:, c], lambda r: dirichlet_precond(sys, r), tol, maxit, x0)
        lam[:, c] = x
        its.append(it); rel.append(hist[-1]); kap.append(lanczos_condition(al, be))
    # Eq. (8): a_p = C F^-1 (d - G^T lam)
    if sys.n_gp:
        p = np.linalg.solve(op.F, op.d - op.G.T @ lam)
    else:
        p = np.zeros((0, nr))
    # Eq. (9): a_r = K_rr^-1 (j_r - K_rp a_p - B_r^T lam)
    a_r = []
    for s in sys.subs:
        ap = p[s.Cidx]
        a_r.append(s.lu.solve(s.jr - s.Krp @ ap - _BrT(s, lam)))
    # global field: lowest subdomain's copy, primal from p, tree/Dirichlet zero
    a = np.zeros((sys.mesh.nedge, nr))
    done = np.zeros(sys.mesh.nedge, bool)
    for s, ar in zip(sys.subs, a_r):
        new = ~done[s.r_ids]
        a[s.r_ids[new]] = ar[new]
        done[s.r_ids] = True
    a[sys.topo.primal_edges] = p
    jump = np.zeros((sys.m_r, nr))
    for s, ar in zip(sys.subs, a_r):
        _Br_add(s, ar, jump)
    jump_rel = np.linalg.norm(jump) / max(np.linalg.norm(a), 1e-300)
    return DPSolution(lam=lam, p=p, a_r=a_r, a=a, iters=its, relres=rel, kappa=kap, jump=jump_rel)
