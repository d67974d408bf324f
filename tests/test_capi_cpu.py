"""C-ABI library: loads without a GPU, exports every declared entry point, and its
host-side gauge (Sec. 2.2) and DOF classes equal the oracle's."""
import ctypes
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
                              sub_of_patch=wl.block_partition((4, 4, 2), (2, 2, 1)))]


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
