"""Facets, wire basket, Kruskal tree-cotree gauge and DOF classes (oracle, test
infrastructure).

Sec. 2 (facets, wire basket), Sec. 2.2 (tree-cotree gauging, primal selection),
Fig. "weights" (edge weights 1-5).

Readings (the paper is underspecified here):
  * An interface facet is the union of the closed patch-facets shared by two
    subdomains k and l (one facet per pair; Sec. 2 makes each interface a facet).
  * Dirichlet facets of a subdomain: connected components of its boundary
    patch-facets with the same outward label (direction, side) of the glued
    control net. This keeps two boundary patch-facets of one patch that meet along a
    segment in separate facets, as Sec. 2 requires.
  * Wire basket (mesh-edge reading: the edges lying where facets meet): edges in
    the closure of two or more facets of one subdomain, plus every edge shared
    by more than two subdomains.
  * Weights: the first matching rule of Fig. "weights" wins; Kruskal processes
    edges by the key (weight, edge id).
  * The global tree must stay a tree on the Dirichlet boundary (Sec. 2.2). If the
    weight order fails that, Kruskal is rerun with every boundary edge ordered
    before the weight-2 edges.
  * Primal DOFs = cotree edges of weight 2 (Sec. 2.2). Patch-interface DOFs inside
    a subdomain are assembled conformingly and add no coarse DOFs.
  * Dual DOFs: remaining edges on an interface; each lies in exactly two
    subdomains. B_r has +1 in the lower subdomain id and -1 in the other.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List

import numpy as np

from . import discretise as dz


class UnionFind:
    def __init__(self, n):
        self.parent = list(range(n))

    def find(self, x):
        root = x
        while self.parent[root] != root:
            root = self.parent[root]
        while self.parent[x] != root:
            self.parent[x], x = root, self.parent[x]
        return root

    def union(self, a, b) -> bool:
        ra, rb = self.find(a), self.find(b)
        if ra == rb:
            return False
        self.parent[rb] = ra
        return True


def _patch_face_edges(prob, mesh, q, d, side):
    """Global ids of the edges in the closure of face (d, side) of patch q."""
    a = dz.patch_abc(prob, q)
    p = prob.p
    n = [prob.nspan[e][a[e]] for e in range(3)]
    st = [mesh.starts[e][a[e]] for e in range(3)]
    out = []
    for de in range(3):
        if de == d:
            continue
        ext = [n[e] + p - (1 if e == de else 0) for e in range(3)]
        rng = [np.arange(ext[e]) for e in range(3)]
        rng[d] = np.array([0 if side == 0 else n[d] + p - 1])
        k, j, i = np.meshgrid(rng[2], rng[1], rng[0], indexing="ij")
        gi = st[0] + i.ravel()
        if mesh.periodic0:
            gi = gi % mesh.N[0]
        out.append(mesh.edge_id(de, gi, st[1] + j.ravel(), st[2] + k.ravel()))
    return np.concatenate(out)


def _neighbour(prob, q, d, side):
    a = list(dz.patch_abc(prob, q))
    a[d] += 1 if side == 1 else -1
    if d == 0 and prob.periodic0:
        a[0] %= prob.npatch[0]
    elif not (0 <= a[d] < prob.npatch[d]):
        return None
    return dz.patch_index(prob, *a)


@dataclasses.dataclass
class Topology:
    nsub: int
    sub_edges: List[np.ndarray]        # sorted global edge ids per subdomain
    mult: np.ndarray                   # subdomains containing each edge
    dirichlet: np.ndarray              # bool per edge
    weight: np.ndarray                 # 1..5 per edge
    tree: np.ndarray                   # bool per edge
    tree_rerun: bool
    primal_edges: np.ndarray           # sorted global ids
    dual_edges: np.ndarray             # sorted global ids
    # per subdomain
    V: List[np.ndarray]                # global ids of r_V (sorted)
    I: List[np.ndarray]                # global ids of r_I (sorted)
    P: List[np.ndarray]                # global ids of primal (sorted)
    dual_of_I: List[np.ndarray]        # global dual index of each I dof
    sign_of_I: List[np.ndarray]        # +1 / -1
    primal_of_P: List[np.ndarray]      # global primal index of each P dof
    nu_edge: List[np.ndarray]          # nu of subdomain k at each I dof (max over its patches)
    wire_basket: np.ndarray            # bool per edge


def build_topology(prob, mesh=None, force_boundary_first=False, reverse_ties=False) -> Topology:
    """``reverse_ties`` breaks weight ties by descending edge id instead (another
    valid spanning tree, used to check gauge invariance)."""
    if mesh is None:
        mesh = dz.build_mesh(prob)
    nsub = prob.nsub
    sub = prob.sub_of_patch
    npt = prob.npatch_total
    pedges = [dz.patch_edges(prob, mesh, q) for q in range(npt)]
    sub_edges = []
    for k in range(nsub):
        sub_edges.append(np.unique(np.concatenate([pedges[q] for q in range(npt) if sub[q] == k])))
    mult = np.zeros(mesh.nedge, np.int64)
    for k in range(nsub):
        mult[sub_edges[k]] += 1
    dirichlet = dz.dirichlet_edges(mesh)

    # --- facets (Sec. 2) and wire basket -------------------------------------
    wire = mult > 2
    for k in range(nsub):
        facets: Dict[object, List[np.ndarray]] = {}
        dir_faces = []  # (q, d, side)
        for q in range(npt):
            if sub[q] != k:
                continue
            for d in range(3):
                for side in (0, 1):
                    nb = _neighbour(prob, q, d, side)
                    if nb is None:
                        dir_faces.append((q, d, side))
                    elif sub[nb] != k:
                        facets.setdefault(("intf", int(sub[nb])), []).append(
                            _patch_face_edges(prob, mesh, q, d, side))
        # Dirichlet facets: connected components per label
        uf = UnionFind(len(dir_faces))
        for i1, (q1, d1, s1) in enumerate(dir_faces):
            for i2, (q2, d2, s2) in enumerate(dir_faces):
                if i2 <= i1 or (d1, s1) != (d2, s2):
                    continue
                a1, a2 = dz.patch_abc(prob, q1), dz.patch_abc(prob, q2)
                diff = [a1[e] - a2[e] for e in range(3)]
                if prob.periodic0:
                    P0 = prob.npatch[0]
                    diff[0] = min(diff[0] % P0, (-diff[0]) % P0)
                if sum(abs(x) for x in diff) == 1 and diff[d1] == 0:
                    uf.union(i1, i2)
        for i, (q, d, side) in enumerate(dir_faces):
            facets.setdefault(("dir", d, side, uf.find(i)), []).append(
                _patch_face_edges(prob, mesh, q, d, side))
        count = np.zeros(mesh.nedge, np.int64)
        for key, lst in facets.items():
            count[np.unique(np.concatenate(lst))] += 1
        wire |= count >= 2

    # --- weights (Fig. "weights"), first matching rule wins ----------------------
    weight = np.full(mesh.nedge, 5, np.int64)
    on_intf = mult >= 2
    rule4 = dirichlet | on_intf
    weight[rule4] = 4
    weight[wire & ~(dirichlet & on_intf) & ~(mult > 2)] = 3
    weight[(mult > 2) & ~(dirichlet & on_intf)] = 2
    weight[dirichlet & on_intf] = 1

    # --- Kruskal (Sec. 2.2) ------------------------------------------------------
    tails, heads = mesh.edge_endpoints()
    bnodes = dz.boundary_nodes(mesh)

    def kruskal(boundary_first):
        key_w = weight.copy()
        if boundary_first:
            # every boundary edge before the weight-2 edges
            key_w = np.where(dirichlet, np.minimum(key_w, 1), key_w)
        tie = -np.arange(mesh.nedge) if reverse_ties else np.arange(mesh.nedge)
        order = np.lexsort((tie, key_w))
        uf = UnionFind(mesh.nnode)
        tree = np.zeros(mesh.nedge, bool)
        for e in order:
            if uf.union(int(tails[e]), int(heads[e])):
                tree[e] = True
        return tree

    def boundary_tree_ok(tree):
        # tree restricted to boundary edges must be a spanning tree of the boundary graph
        nb = int(bnodes.sum())
        return int((tree & dirichlet).sum()) == nb - 1

    tree = kruskal(force_boundary_first)
    rerun = False
    if not boundary_tree_ok(tree):
        tree = kruskal(True)
        rerun = True
    assert int(tree.sum()) == mesh.nnode - 1

    # --- DOF classes ----------------------------------------------------------------
    keep = ~dirichlet & ~tree
    primal_mask = keep & (weight == 2)
    primal_edges = np.flatnonzero(primal_mask)
    dual_mask = keep & ~primal_mask & on_intf
    if np.any(mult[dual_mask] != 2):
        raise RuntimeError("a dual DOF lies in more than two subdomains")
    dual_edges = np.flatnonzero(dual_mask)
    dual_index = -np.ones(mesh.nedge, np.int64)
    dual_index[dual_edges] = np.arange(len(dual_edges))
    primal_index = -np.ones(mesh.nedge, np.int64)
    primal_index[primal_edges] = np.arange(len(primal_edges))

    # lowest subdomain id of each edge
    low = np.full(mesh.nedge, nsub, np.int64)
    for k in range(nsub):
        low[sub_edges[k]] = np.minimum(low[sub_edges[k]], k)

    V, I, P, dual_of_I, sign_of_I, primal_of_P, nu_edge = [], [], [], [], [], [], []
    for k in range(nsub):
        e = sub_edges[k]
        ek = e[keep[e]]
        Pk = ek[primal_mask[ek]]
        Ik = ek[dual_mask[ek]]
        Vk = ek[~primal_mask[ek] & ~dual_mask[ek]]
        V.append(Vk); I.append(Ik); P.append(Pk)
        dual_of_I.append(dual_index[Ik])
        sign_of_I.append(np.where(low[Ik] == k, 1.0, -1.0))
        primal_of_P.append(primal_index[Pk])
        nue = np.zeros(len(Ik))
        for q in range(npt):
            if sub[q] != k:
                continue
            inq = np.isin(Ik, pedges[q])
            nue[inq] = np.maximum(nue[inq], prob.nu[q])
        nu_edge.append(nue)
    return Topology(nsub=nsub, sub_edges=sub_edges, mult=mult, dirichlet=dirichlet,
                    weight=weight, tree=tree, tree_rerun=rerun, primal_edges=primal_edges,
                    dual_edges=dual_edges, V=V, I=I, P=P, dual_of_I=dual_of_I,
                    sign_of_I=sign_of_I, primal_of_P=primal_of_P, nu_edge=nu_edge,
                    wire_basket=wire)
