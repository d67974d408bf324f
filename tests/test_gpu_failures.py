"""Failure paths of the C ABI, with every fault injected from the host.

No device code is made to fault, trap or hang: the waits of the dependency
sweeps are bounded, and a test lowers their poll limit through the library's
testing hook so that they give up; the pivot failure is a negative diagonal
entry written into the factor buffer from the host; the other cases are bad
inputs (a NaN initial guess, an iteration cap). After each failure the same
context, and a fresh one, still solve the problem to the oracle's field.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import discretise as dz, monolithic as mono, topology as tp
from paper_2501_04340_gb300 import workloads as wl


@pytest.fixture(scope="module")
def ieti():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_04340_gb300 import ieti as m
    return m


@pytest.fixture(scope="module")
def case():
    rng = np.random.default_rng(4)
    prob = wl.unit_cube(3, (4, 4, 2), 3, sub_of_patch=wl.block_partition((4, 4, 2), (2, 2, 1)),
                        nu=10.0 ** rng.uniform(0, 3, 32), name="cube32_p3n3_sub8")
    mesh, Kp, jp = dz.assemble_all(prob)
    topo = tp.build_topology(prob, mesh)
    a_ref, _ = mono.solve(mesh, topo, Kp, jp)
    return prob, mesh, a_ref[:, 0]


def _solve_ok(ieti, ctx, prob, mesh, a_ref, prec):
    a = torch.zeros((1, mesh.nedge), dtype=torch.float64, device="cuda")
    info = ieti.ieti_solve(ctx, a, tol=1e-11, maxit=600, tol_field=1e-12 if prec else 0.0)
    assert info.converged == 1
    ag = a.cpu().numpy()[0]
    assert np.linalg.norm(ag - a_ref) <= 1e-8 * np.linalg.norm(a_ref)


@pytest.mark.parametrize("prec", [0, 1])
def test_iteration_cap_gives_no_convergence_with_info(ieti, case, prec):
    prob, mesh, a_ref = case
    ctx = ieti.ieti_create(prob)
    try:
        ieti.ieti_assemble(ctx)
        ieti.ieti_factor(ctx, prec)
        a = torch.zeros((1, mesh.nedge), dtype=torch.float64, device="cuda")
        with pytest.raises(ieti.IetiError, match="NO_CONVERGENCE"):
            ieti.ieti_solve(ctx, a, tol=1e-11, maxit=3, tol_field=1e-12 if prec else 0.0)
        info = ieti.ieti_solve(ctx, a, tol=1e-11, maxit=3, tol_field=1e-12 if prec else 0.0,
                               allow_no_convergence=True)
        assert info.converged == 0
        assert info.relres > 1e-11 and np.isfinite(info.relres)
        if prec == 0:
            assert info.iterations == 3 and info.refinement_steps == 1
        else:
            assert info.refinement_steps == 16 and info.iterations <= 16 * 3
            assert info.fp64_fallback == 0     # the inner PCG was capped: not a precision failure
            assert info.global_relres > 1e-12
        _solve_ok(ieti, ctx, prob, mesh, a_ref, prec)
    finally:
        ieti.ieti_destroy(ctx)


def test_nan_initial_guess_is_refused(ieti, case):
    prob, mesh, a_ref = case
    ctx = ieti.ieti_create(prob)
    try:
        ieti.ieti_assemble(ctx)
        ieti.ieti_factor(ctx, ieti.IETI_FP64)
        m = ieti.ieti_query(ctx)["m_r"]
        lam0 = torch.zeros((1, m), dtype=torch.float64, device="cuda")
        lam0[0, m // 2] = float("nan")
        a = torch.zeros((1, mesh.nedge), dtype=torch.float64, device="cuda")
        with pytest.raises(ieti.IetiError, match="INVALID_ARG.*NaN"):
            ieti.ieti_solve(ctx, a, lam0=lam0, tol=1e-11)
        lam0[0, m // 2] = float("inf")
        with pytest.raises(ieti.IetiError, match="INVALID_ARG"):
            ieti.ieti_solve(ctx, a, lam0=lam0, tol=1e-11)
        _solve_ok(ieti, ctx, prob, mesh, a_ref, 0)
    finally:
        ieti.ieti_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
def test_forced_pivot_failure_names_the_subdomain(ieti, case, prec):
    prob, mesh, a_ref = case
    ctx = ieti.ieti_create(prob)
    try:
        ieti.ieti_assemble(ctx)
        ieti.ieti_debug_set(ctx, ieti.IETI_DEBUG_PIVOT_FAULT, 5)
        with pytest.raises(ieti.IetiError, match="SINGULAR_LOCAL.*subdomain 5"):
            ieti.ieti_factor(ctx, prec)
        ieti.ieti_debug_set(ctx, ieti.IETI_DEBUG_PIVOT_FAULT, -1)
        ieti.ieti_factor(ctx, prec)
        _solve_ok(ieti, ctx, prob, mesh, a_ref, prec)
        with pytest.raises(ieti.IetiError, match="INVALID_ARG"):
            ieti.ieti_debug_set(ctx, ieti.IETI_DEBUG_PIVOT_FAULT, 8)
    finally:
        ieti.ieti_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
def test_timed_out_sweep_waits_return_timeout(ieti, case, prec):
    """A poll limit of zero makes the first wait on an unpublished block give
    up: the factorisation (multi-column W and Phi solves) and the solve
    (single-column sweeps) report TIMEOUT, and both work again once the limit
    is restored; a fresh context is unaffected."""
    prob, mesh, a_ref = case
    ctx = ieti.ieti_create(prob)
    try:
        ieti.ieti_assemble(ctx)
        ieti.ieti_debug_set(ctx, ieti.IETI_DEBUG_WAIT_POLLS, 0)
        with pytest.raises(ieti.IetiError, match="TIMEOUT"):
            ieti.ieti_factor(ctx, prec)
        ieti.ieti_debug_set(ctx, ieti.IETI_DEBUG_WAIT_POLLS, -1)
        ieti.ieti_factor(ctx, prec)
        ieti.ieti_debug_set(ctx, ieti.IETI_DEBUG_WAIT_POLLS, 0)
        a = torch.zeros((1, mesh.nedge), dtype=torch.float64, device="cuda")
        with pytest.raises(ieti.IetiError, match="TIMEOUT"):
            ieti.ieti_solve(ctx, a, tol=1e-11, maxit=50, tol_field=1e-12 if prec else 0.0)
        ieti.ieti_debug_set(ctx, ieti.IETI_DEBUG_WAIT_POLLS, -1)
        _solve_ok(ieti, ctx, prob, mesh, a_ref, prec)
    finally:
        ieti.ieti_destroy(ctx)
    ctx = ieti.ieti_create(prob)
    try:
        ieti.ieti_assemble(ctx)
        ieti.ieti_factor(ctx, prec)
        _solve_ok(ieti, ctx, prob, mesh, a_ref, prec)
    finally:
        ieti.ieti_destroy(ctx)
