"""The learned warm start on a reduced instance family: what the trained
network gains over PCG from a zero guess, and that the guess never changes
the answer.

Family: unit cube, 4 x 4 x 4 affine patches (p = 2, 2 spans per patch and
direction), 8 subdomains of 2 x 2 x 2 patches, per-patch nu = 10^(3u),
u ~ U(0, 1), and 16 Fourier source coefficients ~ N(0, 1). Training data: 256
sampled nu, each solved for the 16 unit sources (FP64 factors, tol 1e-10);
held out: 32 instances with fresh nu and coefficients, solved to 1e-8.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_04340_gb300 import workloads as wl

NTR, NTE = 256, 32


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_04340_gb300 import ieti, warmstart as ws
    fam = wl.warmstart_family(NTR + NTE, seed=21)
    tr, te = np.arange(NTR), np.arange(NTR, NTR + NTE)
    ctx16 = ws.basis_context(fam)
    basis = ws.solve_basis(ctx16, fam, tr, tol=1e-10)
    ieti.ieti_destroy(ctx16)
    m, loss = ws.train(fam, tr, basis, hidden=256, batch=64, epochs=300, lr=1e-3, decay=0.995)
    ctx1 = ws.instance_context(fam)
    yield ieti, ws, fam, tr, te, basis, m, loss, ctx1
    ieti.ieti_mlp_destroy(m)
    ieti.ieti_destroy(ctx1)


def test_training_data_converged(setup):
    ieti, ws, fam, tr, te, basis, m, loss, ctx1 = setup
    assert np.all(basis.relres <= 1e-10)
    assert np.isfinite(loss)


def test_warm_start_saves_iterations_and_keeps_the_answer(setup):
    ieti, ws, fam, tr, te, basis, m, loss, ctx1 = setup
    lam0 = ws.predict(m, fam, te)
    zero = ws.solve_instances(ctx1, fam, te, tol=1e-8, keep_fields=True)
    warm = ws.solve_instances(ctx1, fam, te, tol=1e-8, lam0=lam0, keep_fields=True)
    exact = ws.solve_instances(ctx1, fam, te, tol=1e-12)
    err0 = (torch.linalg.norm(lam0 - exact.lam[:, 0], dim=1) / torch.linalg.norm(exact.lam[:, 0], dim=1))
    print(f"\nwarm start on {NTE} held-out instances: PCG iterations {zero.iterations.mean():.2f} (zero guess) "
          f"-> {warm.iterations.mean():.2f} (network), mean relative error of lambda0 {err0.mean().item():.3f}")
    assert np.all(zero.relres <= 1e-8) and np.all(warm.relres <= 1e-8)
    assert warm.iterations.mean() <= zero.iterations.mean() - 1.0
    assert err0.mean().item() < 1.0
    d = torch.linalg.norm(warm.fields - zero.fields) / torch.linalg.norm(zero.fields)
    assert d.item() <= 1e-6


def test_a_bad_guess_only_costs_iterations(setup):
    """PCG from a useless guess (1e3 times the scale of the multipliers, random
    directions) still meets the same stopping test and returns the same field."""
    ieti, ws, fam, tr, te, basis, m, loss, ctx1 = setup
    idx = te[:4]
    exact = ws.solve_instances(ctx1, fam, idx, tol=1e-12, keep_fields=True)
    g = torch.Generator(device="cpu").manual_seed(3)
    scale = exact.lam.abs().max().item()
    bad = (torch.randn(exact.lam[:, 0].shape, generator=g, dtype=torch.float64) * 1e3 * scale).cuda()
    res = ws.solve_instances(ctx1, fam, idx, tol=1e-8, lam0=bad, keep_fields=True)
    assert np.all(res.relres <= 1e-8)
    d = torch.linalg.norm(res.fields - exact.fields) / torch.linalg.norm(exact.fields)
    assert d.item() <= 1e-6
