"""The solve of the bench workload against the stored oracle field.

Workload: the unit cube in 4 x 4 x 4 patches, 16 subdomains of 2 x 2 x 1
patches, p = 3, 8 spans, per-patch nu log-uniform in [1, 1e3] (seed 2), the
sine source. tests/golden/cube64_p3n8_sub16.npz holds the FP64 oracle solve
of Eqs. (7)-(9) (PCG to 1e-13, written by tests/golden/make_golden.py).

Checks, for the plain FP64 path and the FP32 path with FP64 refinement, both
in the launch configuration the bench times (interface tolerance 1e-8, field
tolerance 1e-8 for the refinement) and at tight tolerances:
  ||a - a_oracle|| <= 1e-8 ||a_oracle||  and  ||B(a) - B(a_oracle)||_L2 <= 1e-8 ||B(a_oracle)||_L2,
with B = curl a evaluated on the device (pinned against the oracle's
quadrature in test_gpu_flux.py) and ||B(a_oracle)|| per patch from the file.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2501_04340_gb300 import workloads as wl

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "cube64_p3n8_sub16.npz")


@pytest.fixture(scope="module")
def ieti():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_04340_gb300 import ieti as m
    return m


@pytest.fixture(scope="module")
def gold():
    g = np.load(GOLD)
    a = np.zeros(int(g["nedge"]))
    a[g["a_idx"]] = g["a_val"][:, 0]
    return a, g["nB"][0]


@pytest.fixture(scope="module")
def ctx_by_prec(ieti):
    prob = wl.cube64_p3n8_sub16()
    out = {}
    for prec in (ieti.IETI_FP64, ieti.IETI_FP32_IR):
        c = ieti.ieti_create(prob)
        ieti.ieti_assemble(c)
        ieti.ieti_factor(c, prec)
        out[prec] = c
    yield prob, out
    for c in out.values():
        ieti.ieti_destroy(c)


@pytest.mark.parametrize("prec,tol,tol_field", [(0, 1e-11, 0.0), (1, 1e-8, 1e-8), (1, 1e-10, 1e-10), (0, 1e-10, 0.0)])
def test_field_and_flux_match_the_oracle(ieti, gold, ctx_by_prec, prec, tol, tol_field):
    """The FP32 factors of this workload are inside their regime: the
    refinement never falls back to FP64 here."""
    a_ref, nB_ref = gold
    prob, ctxs = ctx_by_prec
    ctx = ctxs[prec]
    a = torch.zeros((1, len(a_ref)), dtype=torch.float64, device="cuda")
    info = ieti.ieti_solve(ctx, a, tol=tol, maxit=2000, tol_field=tol_field)
    assert info.converged == 1 and info.fp64_fallback == 0
    ag = a.cpu().numpy()[0]
    err_a = np.linalg.norm(ag - a_ref) / np.linalg.norm(a_ref)
    assert err_a <= 1e-8, err_a
    d = torch.tensor((ag - a_ref)[None, :], dtype=torch.float64, device="cuda")
    dB2, _ = ieti.ieti_eval_B(ctx, d, prob.npatch_total)
    nB2, _ = ieti.ieti_eval_B(ctx, a, prob.npatch_total)
    nB = np.sqrt((nB_ref ** 2).sum())
    assert np.sqrt(dB2.sum()) <= 1e-8 * nB
    # per patch: the device norm of the GPU field equals the oracle's norm of its field
    assert np.abs(np.sqrt(nB2[0]) - nB_ref).max() <= 1e-8 * nB_ref.max()
