"""C-ABI library: loads without a GPU, exports every declared entry point, and its
host-side gauge (Sec. 2.2) and DOF classes equal the oracle's."""
import ctypes
import dataclasses
import os

import numpy as np
import pytest

from oracle import topology as tp
from paper_2501_04340_gb300 import workloads as wl

ieti = pytest.importorskip("paper_2501_04340_gb300.ieti")


def test_library_exports_every_declared_symbol():
    lib = ctypes.CDLL(ieti.LIB_PATH)
    syms = ieti.header_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s


CASES = [lambda: wl.cube8_p2n4(), lambda: wl.small_cases()[1], lambda: wl.small_cases()[2],
         lambda: wl.small_cases()[3], lambda: wl.cube64_p3n8_sub16(),
         lambda: wl.unit_cube(2, (4, 4, 2), [[1, 2, 1, 3], [2, 1, 1, 2], [2, 1]],
                              sub_of_patch=wl.block_partition((4, 4, 2), (2, 2, 1))),
         lambda: wl.machine_annulus(n_ang=12, n_ax=1, spans=2, nrhs=2),
         lambda: wl.machine_annulus(nrhs=1)]


@pytest.mark.parametrize("make", CASES)
def test_host_gauge_equals_oracle(make):
    prob = make()
    topo = tp.build_topology(prob)
    ctx = ieti.ieti_create_host(prob)
    try:
        q = ieti.ieti_query(ctx)
        assert q["m_r"] == len(topo.dual_edges) and q["n_gp"] == len(topo.primal_edges)
        assert q["n_gauged"] == int((~topo.dirichlet & ~topo.tree).sum())
        assert np.array_equal(ieti.ieti_get_dofmap(ctx, 0).astype(bool), topo.tree)
        assert np.array_equal(ieti.ieti_get_dofmap(ctx, 1), topo.weight)
        assert np.array_equal(ieti.ieti_get_dofmap(ctx, 2), topo.primal_edges)
        assert np.array_equal(ieti.ieti_get_dofmap(ctx, 3), topo.dual_edges)
        for k in range(topo.nsub):
            # r_V DOFs: the same set, in the library's banded order (by control index)
            assert np.array_equal(np.sort(ieti.ieti_get_dofmap(ctx, 4, k)), topo.V[k])
            assert np.array_equal(ieti.ieti_get_dofmap(ctx, 5, k), topo.I[k])
            assert np.array_equal(ieti.ieti_get_dofmap(ctx, 6, k), topo.P[k])
            assert np.array_equal(ieti.ieti_get_dofmap(ctx, 7, k), topo.sign_of_I[k].astype(np.int64))
    finally:
        ieti.ieti_destroy(ctx)


def test_rejects_non_simply_connected_subdomain():
    # a ring of 8 patches around the centre column of a 3x3x1 grid
    sub = np.ones(9, np.int32)
    sub[4] = 0
    prob = wl.unit_cube(1, (3, 3, 1), 1, sub_of_patch=sub)
    with pytest.raises(ieti.IetiError, match="NOT_SIMPLY_CONNECTED"):
        ieti.ieti_create_host(prob)


def test_rejects_bad_degree_and_sizes():
    prob = wl.unit_cube(1, (2, 1, 1), 1)
    prob.p = 5
    with pytest.raises(ieti.IetiError, match="INVALID_ARG"):
        ieti.ieti_create_host(prob)
    prob = wl.unit_cube(1, (2, 1, 1), 1)
    prob.nrhs = 0
    with pytest.raises(ieti.IetiError, match="INVALID_ARG"):
        ieti.ieti_create_host(prob)


def test_device_entry_points_refuse_host_context():
    ctx = ieti.ieti_create_host(wl.cube8_p2n4(spans=1))
    try:
        with pytest.raises(ieti.IetiError, match="STATE"):
            ieti.ieti_assemble(ctx)
    finally:
        ieti.ieti_destroy(ctx)


def _decode_edges(prob, e):
    """(direction, i, j, k) of global edge ids: direction blocks one after the
    other, i fastest; direction d has one edge fewer along d (not periodic)."""
    N = prob.grid_shape()
    ext, off = [], [0]
    for d in range(3):
        x = list(N)
        if not (d == 0 and prob.periodic0):
            x[d] -= 1
        ext.append(x)
        off.append(off[-1] + x[0] * x[1] * x[2])
    d = np.searchsorted(np.array(off[1:]), e, side="right")
    r = e - np.array(off)[d]
    e0 = np.array([ext[q][0] for q in d])
    e1 = np.array([ext[q][1] for q in d])
    return d, r % e0, (r // e0) % e1, r // (e0 * e1)


@pytest.mark.parametrize("make", [lambda: wl.cube64_p3n8_sub16(), lambda: wl.small_cases()[2]])
def test_interior_dofs_in_banded_order(make):
    """The r_V DOFs of every subdomain are ordered lexicographically in the
    control index of their edge (longest axis outermost, shortest innermost),
    then by direction: the order that keeps K_rr banded for the factor."""
    prob = make()
    ctx = ieti.ieti_create_host(prob)
    try:
        for k in range(prob.nsub):
            V = ieti.ieti_get_dofmap(ctx, 4, k)
            if len(V) < 2:
                continue
            d, i, j, kk = _decode_edges(prob, V)
            c = np.stack([i, j, kk])
            ext = c.max(axis=1) - c.min(axis=1)
            ax = sorted(range(3), key=lambda a: -ext[a])   # stable: ties keep axis order
            key = np.stack([c[ax[0]], c[ax[1]], c[ax[2]], d, V]).T
            assert all(tuple(key[q]) < tuple(key[q + 1]) for q in range(len(V) - 1)), k
    finally:
        ieti.ieti_destroy(ctx)


def test_uneven_partition_of_the_512_patch_cube():
    """The uneven 64-subdomain partition of the 512-patch cube (the batching
    workload): sizes within 4..12 patches, every subdomain simply connected
    (the library's own check accepts it), and the host DOF classes split every
    subdomain's edges."""
    prob = wl.cube512_p3_uneven64(nrhs=1)
    size = np.bincount(prob.sub_of_patch, minlength=64)
    assert prob.nsub == 64 and size.min() >= 4 and size.max() <= 12 and size.sum() == 512
    assert size.min() < size.max()   # uneven
    for k in range(64):
        assert wl.is_simply_connected_union((8, 8, 8), np.flatnonzero(prob.sub_of_patch == k))
    ctx = ieti.ieti_create_host(prob)
    try:
        q = ieti.ieti_query(ctx)
        assert q["nsub"] == 64 and q["m_r"] > 0 and q["n_gp"] > 0
        nI = [len(ieti.ieti_get_dofmap(ctx, 5, k)) for k in range(64)]
        nV = [len(ieti.ieti_get_dofmap(ctx, 4, k)) for k in range(64)]
        assert min(nV) > 0 and min(nI) > 0 and max(nI) == q["max_nI"]
    finally:
        ieti.ieti_destroy(ctx)


def test_affine_flag_is_checked():
    """The Kronecker assembly is exact only for axis-aligned boxes: a claim of
    affine maps on any other control net is rejected, whatever the weights."""
    box = wl.unit_cube(2, (2, 1, 1), [[2, 3], [2], [1]])
    ieti.ieti_destroy(ieti.ieti_create_host(box))
    bent = wl.unit_cube(2, (2, 1, 1), [[2, 3], [2], [1]])
    bent.ctrl[1, 1, 2, 0] += 0.01          # one interior control point moved: unit weights, not a box
    with pytest.raises(ieti.IetiError, match="INVALID_ARG.*affine"):
        ieti.ieti_create_host(bent)
    bent.affine = False
    ieti.ieti_destroy(ieti.ieti_create_host(bent))
    ring = wl.machine_annulus(n_ang=12, n_ax=1, spans=2, nrhs=1)
    assert not ring.affine
    ring.affine = True
    with pytest.raises(ieti.IetiError, match="INVALID_ARG"):
        ieti.ieti_create_host(ring)


@pytest.mark.parametrize("p,spans,nsub", [(1, 2, 3), (2, 1, 5), (3, 1, 2)])
def test_host_boundary_data_equals_oracle(p, spans, nsub):
    """The library's boundary L2 projection of the tangential trace of A_ana
    (IETI_SOURCE_TRIG, computed on the host in ieti_create) equals the oracle's."""
    from oracle import boundary as bd, discretise as dz
    prob = wl.paper_cube(p, spans, nsub=nsub)
    mesh = dz.build_mesh(prob)
    want = bd.boundary_projection(prob, mesh, bd.manufactured_A)
    ctx = ieti.ieti_create_host(prob)
    try:
        got = ieti.ieti_get_boundary_data(ctx)
    finally:
        ieti.ieti_destroy(ctx)
    assert got.shape == want.shape
    assert np.array_equal(got != 0, want != 0)
    assert np.abs(got - want).max() <= 1e-11 * np.abs(want).max()


def test_homogeneous_kinds_have_no_boundary_data():
    ctx = ieti.ieti_create_host(wl.cube8_p2n4(spans=1))
    try:
        assert ieti.ieti_get_boundary_data(ctx).size == 0
    finally:
        ieti.ieti_destroy(ctx)


def test_rejects_source_parameters_that_do_not_fit_the_kind():
    base = wl.cube8_p2n4(spans=1)
    bad = [base.with_params(source_params=[1.0], nrhs=2),                      # sine: 2 amplitudes needed
           dataclasses.replace(base, source_kind=wl.SOURCE_PATCHWISE, source_params=np.zeros(3 * 8 - 1)),
           dataclasses.replace(base, source_kind=wl.SOURCE_FOURIER, source_params=np.array([2.0] + [0.0] * 9)),
           dataclasses.replace(base, source_kind=7),
           # the manufactured Dirichlet data needs affine boxes
           dataclasses.replace(wl.paper_cube(1, 1), affine=False)]
    for prob in bad:
        with pytest.raises(ieti.IetiError, match="INVALID_ARG"):
            ieti.ieti_create_host(prob)


@pytest.mark.parametrize("make", [lambda: wl.paper_cube(2, 2), lambda: wl.paper_cube(1, 2, nsub=5, layout="snake"),
                                  lambda: wl.paper_cube(3, 1, nsub=12, layout="snake")])
def test_host_gauge_equals_oracle_on_the_paper_cube(make):
    """The 27-patch cube of Sec. 3 with the layouts of the experiments: the same
    tree, primal and dual sets on the host as in the oracle."""
    prob = make()
    topo = tp.build_topology(prob)
    ctx = ieti.ieti_create_host(prob)
    try:
        assert np.array_equal(ieti.ieti_get_dofmap(ctx, 0).astype(bool), topo.tree)
        assert np.array_equal(ieti.ieti_get_dofmap(ctx, 2), topo.primal_edges)
        assert np.array_equal(ieti.ieti_get_dofmap(ctx, 3), topo.dual_edges)
    finally:
        ieti.ieti_destroy(ctx)


def test_coarse_size_of_the_three_columns_does_not_depend_on_h_and_p():
    """Sec. 3, Experiment 1: one interior line of patch edges is shared by the
    three subdomains; all of its edges but one join the tree, so n_gp = 1 for
    every mesh size and degree (and 0 for three slabs, which share no line)."""
    for p in (1, 2, 3):
        for n in (1, 2, 3):
            for layout, want in (("columns", 1), ("snake", 0)):
                ctx = ieti.ieti_create_host(wl.paper_cube(p, n, layout=layout))
                try:
                    assert ieti.ieti_query(ctx)["n_gp"] == want, (p, n, layout)
                finally:
                    ieti.ieti_destroy(ctx)
