"""Gauged monolithic direct solve (oracle, test infrastructure).

Eq. (3) K_g a_g = j_g restricted to the DOFs that are neither Dirichlet
(n x A = 0, Sec. 2) nor tree edges of the same global spanning tree (Sec. 2.2:
tree edges are the undetermined DOFs, set to zero). The dual-primal method of
Eqs. (7)-(9) reaches exactly this solution, so it is the parity target.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def global_matrix(Kpatch, jpatch):
    K = Kpatch[0]
    j = jpatch[0]
    for Kq, jq in zip(Kpatch[1:], jpatch[1:]):
        K = K + Kq
        j = j + jq
    return K.tocsr(), j


def solve(mesh, topo, Kpatch, jpatch):
    """Returns (a (nedge x nrhs), keep mask)."""
    K, j = global_matrix(Kpatch, jpatch)
    keep = ~topo.dirichlet & ~topo.tree
    idx = np.flatnonzero(keep)
    Kk = K[idx][:, idx].tocsc()
    lu = spla.splu(Kk)
    a = np.zeros((mesh.nedge, j.shape[1]))
    a[idx] = lu.solve(j[idx])
    return a, keep
