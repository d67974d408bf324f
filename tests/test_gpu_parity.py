"""GPU parity: every step of the CUDA path against the FP64 oracle, element by
element on seeded synthetic problems (small cases span several 64-wide panels
and ragged tails).

Tolerances (relative, max-norm unless stated):
  * assembly (FP64 on both sides, different summation order): 1e-12;
  * FP64 factorisation products (S_rIrI, its inverse, S_Pi, F_DP, M_D^-1): 1e-9
    (condition numbers of the local blocks are below 1e4 here);
  * FP32 operators: max(2e-3, kappa_max u_32), with kappa_max the largest
    condition number of the local blocks K_rr^(k) (dense eigenvalues in the
    oracle) and u_32 = 2^-24: the first-order error of an inverse from an FP32
    Cholesky factor; a case with kappa_max u_32 >= 1 is outside the FP32
    regime and only its solve is checked (the refinement falls back to FP64);
  * the field a and the flux B = curl a against the monolithic oracle solve:
    1e-8 in the 2-norm, for both precisions (FP32 through FP64 refinement).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import discretise as dz, topology as tp, fetidp as fd, monolithic as mono, post
from paper_2501_04340_gb300 import workloads as wl


@pytest.fixture(scope="module")
def ieti():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_04340_gb300 import ieti as m
    return m


def _ragged():
    return wl.unit_cube(3, (2, 2, 1), [[2, 3], [3, 2], [3]], sub_of_patch=np.array([0, 1, 0, 2], np.int32),
                        nu=[1.0, 30.0, 2.0, 500.0], nrhs=2, source_params=[1.0, -2.0])


def _cube32_p3n3_sub8():
    """16 panels per subdomain, nu jumps up to 1e3, 8 subdomains of 2 x 2 x 1 patches."""
    rng = np.random.default_rng(4)
    return wl.unit_cube(3, (4, 4, 2), 3, sub_of_patch=wl.block_partition((4, 4, 2), (2, 2, 1)),
                        nu=10.0 ** rng.uniform(0, 3, 32), name="cube32_p3n3_sub8", nrhs=2,
                        source_params=[1.0, -0.5])


def _cube18_p3_mixed():
    """Mixed spans 3/4 per slab, uneven subdomains of 1 to 4 patches (up to 23 panels), nu jumps."""
    rng = np.random.default_rng(6)
    P = (3, 3, 2)
    sub = np.array([min(a, 1) + 2 * (b // 2) + 4 * c for c in range(2) for b in range(3) for a in range(3)])
    return wl.unit_cube(3, P, [[3, 4, 3], [4, 3, 4], [3, 4]], sub_of_patch=np.unique(sub, return_inverse=True)[1],
                        nu=10.0 ** rng.uniform(0, 3, 18), name="cube18_p3_mixed", nrhs=1)


CASES = {
    "cube8_p2n4": lambda: wl.cube8_p2n4(),
    "cube8_p1n2": lambda: wl.small_cases()[1],
    "cube12_p2_mixed": lambda: wl.small_cases()[3],
    "ragged_p3": _ragged,
    "cube32_p3n3_sub8": _cube32_p3n3_sub8,
    "cube18_p3_mixed": _cube18_p3_mixed,
    # curved, periodic: the NURBS ring (exact 30-degree arcs), air / iron nu jump 1e3, slot currents
    "ring24_p3n2": lambda: wl.machine_annulus(n_ang=12, n_ax=1, spans=2, nrhs=2),
}

_cache = {}


def oracle_case(name):
    if name not in _cache:
        prob = CASES[name]()
        mesh, Kp, jp = dz.assemble_all(prob)
        topo = tp.build_topology(prob, mesh)
        sysd = fd.build_system(prob, (mesh, Kp, jp), topo)
        a_m, _ = mono.solve(mesh, topo, Kp, jp)
        _cache[name] = (prob, mesh, topo, sysd, a_m)
    return _cache[name]


_kappa = {}


def fp32_tol(name):
    """Tolerance of the FP32 operator checks (module docstring); None if the
    case is outside the FP32 regime."""
    if name not in _kappa:
        sysd = oracle_case(name)[3]
        _kappa[name] = max(np.linalg.cond(s.Krr.toarray()) for s in sysd.subs)
        print(f"{name}: max kappa(K_rr) = {_kappa[name]:.3e}")
    ku = _kappa[name] * 2.0 ** -24
    return None if ku >= 1.0 else max(2e-3, ku)


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("affine", [1, 0])
def test_assembly_blocks(ieti, name, affine):
    prob, mesh, topo, sysd, _ = oracle_case(name)
    prob = prob.with_params()
    if affine and not prob.affine:
        # the Kronecker path is only for boxes: the library refuses the claim
        prob.affine = True
        with pytest.raises(ieti.IetiError, match="INVALID_ARG"):
            ieti.ieti_create(prob)
        return
    prob.affine = bool(affine)
    ctx = ieti.ieti_create(prob)
    try:
        ieti.ieti_assemble(ctx)
        for k, s in enumerate(sysd.subs):
            # the library orders the r_V DOFs for a banded factor; compare in its order
            r_lib = np.concatenate([ieti.ieti_get_dofmap(ctx, 4, k), ieti.ieti_get_dofmap(ctx, 5, k)])
            pos = {int(e): i for i, e in enumerate(s.r_ids)}
            p = np.array([pos[int(e)] for e in r_lib], dtype=np.int64)
            assert np.array_equal(np.sort(p), np.arange(len(s.r_ids)))
            Krr = ieti.ieti_get_block(ctx, 0, k)
            assert rel(Krr, s.Krr.toarray()[np.ix_(p, p)]) < 1e-12
            if len(s.Cidx):
                assert rel(ieti.ieti_get_block(ctx, 1, k), s.Krp[p]) < 1e-12
                assert rel(ieti.ieti_get_block(ctx, 2, k), s.Kpp) < 1e-12
            assert rel(ieti.ieti_get_block(ctx, 3, k), s.jr[p]) < 1e-12
            if len(s.Cidx):
                assert rel(ieti.ieti_get_block(ctx, 4, k), s.jp) < 1e-12
    finally:
        ieti.ieti_destroy(ctx)


def _factored(ieti, name, prec):
    prob, mesh, topo, sysd, a_m = oracle_case(name)
    ctx = ieti.ieti_create(prob)
    ieti.ieti_assemble(ctx)
    ieti.ieti_factor(ctx, prec)
    return ctx, prob, mesh, topo, sysd, a_m


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [0, 1])
def test_schur_blocks_and_coarse(ieti, name, prec):
    tol = 1e-9 if prec == 0 else fp32_tol(name)
    if tol is None:
        pytest.skip("kappa(K_rr) u_32 >= 1: FP32 factors outside their regime")
    ctx, prob, mesh, topo, sysd, _ = _factored(ieti, name, prec)
    try:
        op = fd.InterfaceOperator(sysd)
        for k, s in enumerate(sysd.subs):
            S = s.KII - (s.KIV @ s.KVV_lu.solve(s.KIV.T) if s.nV else 0)
            assert rel(ieti.ieti_get_block(ctx, 5, k), S) < tol
            nI = len(s.Brow)
            E = np.zeros((s.Krr.shape[0], nI)); E[s.nV:] = np.eye(nI)
            Winv = s.lu.solve(E)[s.nV:]
            assert rel(ieti.ieti_get_block(ctx, 6, k), Winv) < tol
        if sysd.n_gp:
            assert rel(ieti.ieti_get_coarse(ctx, sysd.n_gp), -op.F) < tol
    finally:
        ieti.ieti_destroy(ctx)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [0, 1])
def test_apply_F_and_preconditioner(ieti, name, prec):
    tol = 1e-9 if prec == 0 else fp32_tol(name)
    if tol is None:
        pytest.skip("kappa(K_rr) u_32 >= 1: FP32 factors outside their regime")
    ctx, prob, mesh, topo, sysd, _ = _factored(ieti, name, prec)
    try:
        op = fd.InterfaceOperator(sysd)
        m = sysd.m_r
        rng = np.random.default_rng(5)
        for nrhs in (1, 3, 11):
            lam = rng.standard_normal((m, nrhs))
            ref = op(lam)
            refM = fd.dirichlet_precond(sysd, lam)
            lam_d = torch.tensor(lam.T.copy(), dtype=torch.float64, device="cuda")
            y = torch.empty_like(lam_d)
            ieti.ieti_apply_F(ctx, lam_d, y, nrhs)
            assert rel(y.cpu().numpy().T, ref) < tol
            z = torch.empty_like(lam_d)
            ieti.ieti_apply_precond(ctx, lam_d, z, nrhs)
            assert rel(z.cpu().numpy().T, refM) < tol
        # interface right-hand side b = e - G F^-1 d
        b = torch.empty((prob.nrhs, m), dtype=torch.float64, device="cuda")
        ieti.ieti_interface_rhs(ctx, b)
        assert rel(b.cpu().numpy().T, op.rhs()) < tol
    finally:
        ieti.ieti_destroy(ctx)


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", [0, 1])
def test_solve_matches_monolithic_field_and_flux(ieti, name, prec):
    ctx, prob, mesh, topo, sysd, a_m = _factored(ieti, name, prec)
    try:
        a = torch.zeros((prob.nrhs, mesh.nedge), dtype=torch.float64, device="cuda")
        lam = torch.zeros((prob.nrhs, sysd.m_r), dtype=torch.float64, device="cuda")
        # field tolerance 1e-10: above the rounding floor of the FP64 residual on
        # every case (about 1e-11 on cube18_p3_mixed); the criterion is the
        # field and flux against the monolithic oracle below
        info = ieti.ieti_solve(ctx, a, tol=1e-11, maxit=400, tol_field=1e-10, lam_out=lam)
        assert info.converged == 1
        ag = a.cpu().numpy().T
        assert np.linalg.norm(ag - a_m) <= 1e-8 * np.linalg.norm(a_m)
        for r in range(prob.nrhs):
            nB, _ = post.flux_l2(prob, mesh, a_m, rhs=r)
            dB, _ = post.flux_l2(prob, mesh, ag - a_m, rhs=r)
            assert dB <= 1e-8 * nB
        # tree and Dirichlet DOFs are exactly zero
        assert np.all(ag[topo.tree | topo.dirichlet] == 0)
        if prec == 0:
            # one pass without field refinement at the paper's PCG tolerance (1e-6,
            # Sec. 3): the oracle's iteration count and Lanczos estimate of kappa.
            # Reading: on the nu-jump cases the PCG residual history has plateaus
            # near the tolerance (on cube32 it goes 1.7e-6, 1.5e-6, 1.4e-6, 1.7e-6,
            # 1.0e-6), where an operator perturbed at rounding level (kappa(K_rr)
            # u_64 ~ 1e-10 between two factorisations; the oracle itself stops one
            # iteration later under a relative 1e-9 perturbation of F) moves the
            # stopping iteration; the counts must agree within max(2, 10 %)
            info1 = ieti.ieti_solve(ctx, a, tol=1e-6, maxit=400, tol_field=0.0)
            sol = fd.solve(sysd, tol=1e-6)
            assert info1.refinement_steps == 1
            assert abs(info1.iterations - max(sol.iters)) <= max(2, 0.1 * max(sol.iters))
            assert abs(info1.kappa - sol.kappa[0]) <= 0.05 * sol.kappa[0]
    finally:
        ieti.ieti_destroy(ctx)


def test_warm_start_with_exact_multipliers_needs_no_iteration(ieti):
    ctx, prob, mesh, topo, sysd, a_m = _factored(ieti, "cube12_p2_mixed", 0)
    try:
        sol = fd.solve(sysd, tol=1e-13)
        lam0 = torch.tensor(sol.lam.T.copy(), dtype=torch.float64, device="cuda")
        a = torch.zeros((prob.nrhs, mesh.nedge), dtype=torch.float64, device="cuda")
        info = ieti.ieti_solve(ctx, a, lam0=lam0, tol=1e-8)
        assert info.iterations == 0
        assert np.linalg.norm(a.cpu().numpy().T - a_m) <= 1e-8 * np.linalg.norm(a_m)
    finally:
        ieti.ieti_destroy(ctx)


@pytest.mark.parametrize("prec", [0, 1])
def test_many_load_cases_match_the_oracle(ieti, prec):
    """Ten load cases at once take the per-phase PCG loop (more than eight
    columns) and the barrier-synchronised multi-column sweeps; by linearity of
    Eq. (3) in the source, column c equals amplitude_c times the oracle field of
    the unit amplitude, to 1e-8."""
    prob, mesh, topo, sysd, a_m = oracle_case("cube12_p2_mixed")
    amps = np.linspace(-2.0, 3.0, 10)
    probn = prob.with_params(source_params=amps, nrhs=10)
    ctx = ieti.ieti_create(probn)
    try:
        ieti.ieti_assemble(ctx)
        ieti.ieti_factor(ctx, prec)
        a = torch.zeros((10, mesh.nedge), dtype=torch.float64, device="cuda")
        info = ieti.ieti_solve(ctx, a, tol=1e-11, maxit=400, tol_field=1e-12 if prec else 0.0)
        assert info.converged == 1
        ag = a.cpu().numpy().T
        ref = a_m[:, :1] * amps[None, :]
        assert np.linalg.norm(ag - ref) <= 1e-8 * np.linalg.norm(ref)
    finally:
        ieti.ieti_destroy(ctx)


def test_tensor_core_trailing_update_path(ieti):
    """The experimental FP32 trailing update on the tensor cores (split TF32
    products) gives a factor good enough for the FP64 refinement: the field
    matches the monolithic oracle solve to 1e-8, like the CUDA-core update. The
    path is chosen before the first factorisation only."""
    prob, mesh, topo, sysd, a_m = oracle_case("cube12_p2_mixed")
    ctx = ieti.ieti_create(prob)
    try:
        ieti.ieti_debug_set(ctx, ieti.IETI_DEBUG_SYRK_TC, 1)
        ieti.ieti_assemble(ctx)
        ieti.ieti_factor(ctx, 1)
        a = torch.zeros((prob.nrhs, mesh.nedge), dtype=torch.float64, device="cuda")
        info = ieti.ieti_solve(ctx, a, tol=1e-10, maxit=400, tol_field=1e-12)
        assert info.converged == 1
        assert np.linalg.norm(a.cpu().numpy().T - a_m) <= 1e-8 * np.linalg.norm(a_m)
        with pytest.raises(ieti.IetiError, match="STATE"):
            ieti.ieti_debug_set(ctx, ieti.IETI_DEBUG_SYRK_TC, 0)
    finally:
        ieti.ieti_destroy(ctx)


def test_fp64_fallback_of_the_refinement(ieti):
    """The refinement's switch to FP64 factors (taken when FP32 factors stall),
    forced from the host: the solve finishes with FP64 factors, reports it, and
    the field equals the monolithic oracle solve to 1e-8; the context keeps the
    FP64 factors for the next solve."""
    ctx, prob, mesh, topo, sysd, a_m = _factored(ieti, "cube12_p2_mixed", 1)
    try:
        ieti.ieti_debug_set(ctx, ieti.IETI_DEBUG_FP64_FALLBACK, 1)
        a = torch.zeros((prob.nrhs, mesh.nedge), dtype=torch.float64, device="cuda")
        info = ieti.ieti_solve(ctx, a, tol=1e-11, maxit=400, tol_field=1e-10)
        assert info.converged == 1 and info.fp64_fallback == 1
        assert np.linalg.norm(a.cpu().numpy().T - a_m) <= 1e-8 * np.linalg.norm(a_m)
        info2 = ieti.ieti_solve(ctx, a, tol=1e-11, maxit=400, tol_field=1e-10)
        assert info2.converged == 1 and info2.fp64_fallback == 0 and info2.refinement_steps <= 3
        assert np.linalg.norm(a.cpu().numpy().T - a_m) <= 1e-8 * np.linalg.norm(a_m)
    finally:
        ieti.ieti_destroy(ctx)


_uneven = {}


@pytest.mark.parametrize("prec", [0, 1])
def test_uneven_subdomains_with_32_load_cases(ieti, prec):
    """The reduced form of the 512-patch workload: 8 uneven simply connected
    subdomains of 4-12 patches, spans 2-4 per patch slab, p = 3, 32 Fourier load
    cases at once (more than eight columns: the per-phase PCG loop and the
    multi-column sweeps). Every column of the field matches the monolithic
    oracle solve to 1e-8, for FP64 factors and for FP32 factors with FP64
    refinement."""
    if not _uneven:
        prob = wl.cube64_uneven8()
        mesh, Kp, jp = dz.assemble_all(prob)
        topo = tp.build_topology(prob, mesh)
        a_m, _ = mono.solve(mesh, topo, Kp, jp)
        _uneven.update(prob=prob, mesh=mesh, a_m=a_m)
    prob, mesh, a_m = _uneven["prob"], _uneven["mesh"], _uneven["a_m"]
    ctx = ieti.ieti_create(prob)
    try:
        ieti.ieti_assemble(ctx)
        ieti.ieti_factor(ctx, prec)
        a = torch.zeros((32, mesh.nedge), dtype=torch.float64, device="cuda")
        info = ieti.ieti_solve(ctx, a, tol=1e-10, maxit=600, tol_field=1e-10 if prec else 0.0)
        assert info.converged == 1
        ag = a.cpu().numpy().T
        err = np.linalg.norm(ag - a_m, axis=0) / np.linalg.norm(a_m, axis=0)
        assert err.max() <= 1e-8, err.max()
    finally:
        ieti.ieti_destroy(ctx)


def test_fourier_loads_match_the_oracle(ieti):
    """Fourier loads (SOURCE_FOURIER): modes with integer wave numbers up to 8
    come from per-point tables of the axis exponentials, the others (a
    non-integer and a large wave number here) are evaluated directly; both give
    the oracle's load blocks to 1e-12."""
    base = wl.cube8_p2n4()
    sp = [3.0,
          1.0, -2.0, 0.0, 0.3, -0.1, 0.2, 0.05, 0.4, -0.3,
          0.5, 1.0, -1.5, 1.0, 0.0, 0.25, -0.2, 0.1, 0.0,
          9.0, 0.0, -11.0, 0.0, 0.7, 0.0, 0.3, 0.0, 0.2,
          2.0,
          8.0, -8.0, 8.0, 0.1, 0.2, -0.3, 0.0, 0.1, 0.1,
          0.0, 0.0, 1.0, -0.4, 0.6, 0.0, 0.2, 0.1, 0.0]
    prob = wl.unit_cube(2, (2, 2, 2), 4, name="cube8_fourier", source_kind=wl.SOURCE_FOURIER,
                        source_params=sp, nrhs=2)
    mesh, Kp, jp = dz.assemble_all(prob)
    topo = tp.build_topology(prob, mesh)
    sysd = fd.build_system(prob, (mesh, Kp, jp), topo)
    ctx = ieti.ieti_create(prob)
    try:
        ieti.ieti_assemble(ctx)
        for k, s in enumerate(sysd.subs):
            r_lib = np.concatenate([ieti.ieti_get_dofmap(ctx, 4, k), ieti.ieti_get_dofmap(ctx, 5, k)])
            pos = {int(e): i for i, e in enumerate(s.r_ids)}
            p = np.array([pos[int(e)] for e in r_lib], dtype=np.int64)
            assert rel(ieti.ieti_get_block(ctx, 3, k), s.jr[p]) < 1e-12
            if len(s.Cidx):
                assert rel(ieti.ieti_get_block(ctx, 4, k), s.jp) < 1e-12
    finally:
        ieti.ieti_destroy(ctx)


def test_step_graphs_replay_the_direct_steps(ieti):
    """After a directly launched first step shows that the persistent PCG
    applies, the refinement steps run from CUDA graphs of their launch
    sequence (captured once per kind of step). A second solve, every step of it
    replayed, gives the field of the first to rounding (the residual's
    assembled sum uses atomic additions), the oracle's to 1e-8, and the same
    count of kernel launches."""
    prob, mesh, topo, sysd, a_m = oracle_case("cube32_p3n3_sub8")
    ctx = ieti.ieti_create(prob)
    try:
        ieti.ieti_assemble(ctx)
        ieti.ieti_factor(ctx, 1)
        out = []
        for _ in range(2):
            a = torch.zeros((prob.nrhs, mesh.nedge), dtype=torch.float64, device="cuda")
            l0 = ieti.ieti_launch_count(ctx)
            info = ieti.ieti_solve(ctx, a, tol=1e-10, maxit=400, tol_field=1e-10)
            out.append((a.cpu().numpy().T, ieti.ieti_launch_count(ctx) - l0, info))
        (a1, n1, i1), (a2, n2, i2) = out
        assert i1.converged == 1 and i2.converged == 1
        assert np.linalg.norm(a2 - a1) <= 1e-12 * np.linalg.norm(a1)
        assert np.linalg.norm(a2 - a_m) <= 1e-8 * np.linalg.norm(a_m)
        assert i1.refinement_steps == i2.refinement_steps and n1 == n2
    finally:
        ieti.ieti_destroy(ctx)


@pytest.mark.parametrize("name", ["ragged_p3", "cube32_p3n3_sub8", "ring24_p3n2"])
@pytest.mark.parametrize("prec", [0, 1])
def test_apply_F_implicit_matches_the_oracle(ieti, name, prec):
    """F_DP through the local factors (sweeps over the r_I blocks) equals the
    oracle's F_DP like the explicit W_k product does (Eq. (7))."""
    tol = 1e-9 if prec == 0 else fp32_tol(name)
    if tol is None:
        pytest.skip("kappa(K_rr) u_32 >= 1: FP32 factors outside their regime")
    ctx, prob, mesh, topo, sysd, _ = _factored(ieti, name, prec)
    try:
        op = fd.InterfaceOperator(sysd)
        nrhs = prob.nrhs
        lam = np.random.default_rng(7).standard_normal((sysd.m_r, nrhs))
        ref = op(lam)
        lam_d = torch.tensor(lam.T.copy(), dtype=torch.float64, device="cuda")
        y = torch.empty_like(lam_d)
        ieti.ieti_apply_F_implicit(ctx, lam_d, y, nrhs)
        assert rel(y.cpu().numpy().T, ref) < tol
        with pytest.raises(ieti.IetiError, match="INVALID_ARG"):
            ieti.ieti_apply_F_implicit(ctx, lam_d, y, nrhs + 1)
    finally:
        ieti.ieti_destroy(ctx)
