"""Pins of the oracle's tree-cotree gauge and DOF classes (Sec. 2.2, Fig. weights)."""
import numpy as np
import pytest

from oracle import discretise as dz, topology as tp, fetidp as fd
from paper_2501_04340_gb300 import workloads as wl

CASES = [lambda: wl.cube8_p2n4(),
         lambda: wl.unit_cube(1, (2, 2, 2), 2),
         lambda: wl.small_cases()[3],
         lambda: wl.unit_cube(2, (4, 4, 2), 1, sub_of_patch=wl.block_partition((4, 4, 2), (2, 2, 1)))]


def _is_spanning_tree(n, tails, heads, sel):
    uf = tp.UnionFind(n)
    for e in np.flatnonzero(sel):
        if not uf.union(int(tails[e]), int(heads[e])):
            return False
    roots = {uf.find(i) for i in range(n)}
    return len(roots) == 1


@pytest.mark.parametrize("make", CASES)
def test_tree_invariants(make):
    prob = make()
    mesh = dz.build_mesh(prob)
    topo = tp.build_topology(prob, mesh)
    t, h = mesh.edge_endpoints()
    # (i) spanning tree of the whole control mesh
    assert topo.tree.sum() == mesh.nnode - 1
    assert _is_spanning_tree(mesh.nnode, t, h, topo.tree)
    # (ii) restricted to the Dirichlet boundary it is a spanning tree of the boundary graph
    bn = dz.boundary_nodes(mesh)
    bidx = -np.ones(mesh.nnode, np.int64)
    bidx[bn] = np.arange(bn.sum())
    sel = topo.tree & topo.dirichlet
    assert _is_spanning_tree(int(bn.sum()), bidx[t], bidx[h], sel)
    # (iii) interior tree edges = interior nodes (kernel dimension of the gauged system)
    assert (topo.tree & ~topo.dirichlet).sum() == (~bn).sum()


def test_gauged_dof_count_unit_cube_p2():
    """2x2x2 patches, p=2, 4 spans: N=11 control points per direction.
    Non-Dirichlet edges 3 (N-1)(N-2)^2 minus interior nodes (N-2)^3 = 1701."""
    prob = wl.cube8_p2n4()
    mesh = dz.build_mesh(prob)
    topo = tp.build_topology(prob, mesh)
    N = 11
    assert mesh.nedge == 3 * (N - 1) * N * N
    assert (~topo.dirichlet).sum() == 3 * (N - 1) * (N - 2) ** 2
    assert (~topo.dirichlet & ~topo.tree).sum() == 3 * (N - 1) * (N - 2) ** 2 - (N - 2) ** 3 == 1701


@pytest.mark.parametrize("make", CASES)
def test_weight_classes_and_dual_multiplicity(make):
    prob = make()
    mesh = dz.build_mesh(prob)
    topo = tp.build_topology(prob, mesh)
    w = topo.weight
    assert np.all(topo.dirichlet[w == 1]) and np.all(topo.mult[w == 1] >= 2)
    assert np.all(topo.mult[w == 2] > 2) and not np.any(topo.dirichlet[w == 2])
    assert np.all(topo.mult[w == 5] == 1) and not np.any(topo.dirichlet[w == 5])
    # every dual DOF in exactly two subdomains, with opposite signs
    count = np.zeros(len(topo.dual_edges))
    ssum = np.zeros(len(topo.dual_edges))
    for k in range(topo.nsub):
        np.add.at(count, topo.dual_of_I[k], 1)
        np.add.at(ssum, topo.dual_of_I[k], topo.sign_of_I[k])
    assert np.all(count == 2) and np.all(ssum == 0)
    # all weight-2 edges are tree or primal (no multiplier on cross-edges)
    assert np.all(topo.tree[w == 2] | np.isin(np.flatnonzero(w == 2), topo.primal_edges))


@pytest.mark.parametrize("make", CASES)
def test_local_blocks_spd(make):
    """Every K_rr^(k) and K_VV^(k) is SPD after tree and primal removal (Sec. 2.1)."""
    prob = make()
    sysd = fd.build_system(prob)
    for s in sysd.subs:
        A = s.Krr.toarray()
        assert np.linalg.eigvalsh(A).min() > 1e-10 * np.abs(A).max()
        AV = A[:s.nV, :s.nV]
        if s.nV:
            assert np.linalg.eigvalsh(AV).min() > 1e-10 * np.abs(AV).max()


def test_coarse_size_independent_of_h_and_p():
    """n_gp does not depend on the mesh size h or the degree p (Sec. 2.2, Sec. 3)."""
    sizes = set()
    for p, n in [(1, 1), (1, 2), (2, 2), (2, 3), (3, 2)]:
        prob = wl.unit_cube(p, (2, 2, 2), n)
        topo = tp.build_topology(prob)
        sizes.add(len(topo.primal_edges))
    assert len(sizes) == 1
    sizes = set()
    for p, n in [(1, 1), (2, 2), (3, 1)]:
        prob = wl.unit_cube(p, (4, 4, 2), n, sub_of_patch=wl.block_partition((4, 4, 2), (2, 2, 1)))
        sizes.add(len(tp.build_topology(prob).primal_edges))
    assert len(sizes) == 1
