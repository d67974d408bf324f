"""The allocation-free interface product against the library's own
preconditioner: for callers that cannot allocate device memory when they need
the product, the library keeps the scratch in a fixed internal array. Two calls
in a row must both reproduce ieti_apply_precond on the same blocks (FP64, same
tolerance as the other FP64 operator tests)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import fetidp as fd
from paper_2501_04340_gb300 import workloads as wl


def test_noalloc_product_matches_preconditioner_twice():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_04340_gb300 import ieti

    prob = wl.small_cases()[3]                      # 6 subdomains, nu jumps, ragged spans
    sysd = fd.build_system(prob)                    # rho-scaling weights of the same reading
    ctx = ieti.ieti_create(prob)
    try:
        ieti.ieti_assemble(ctx)
        ieti.ieti_factor(ctx, ieti.IETI_FP64)
        dual_edges = ieti.ieti_get_dofmap(ctx, 3)
        m = len(dual_edges)
        nI, blocks, dual, weight = [], [], [], []
        for k in range(sysd.topo.nsub):
            S = ieti.ieti_get_block(ctx, 5, k)
            I_edges = ieti.ieti_get_dofmap(ctx, 5, k)
            sign = ieti.ieti_get_dofmap(ctx, 7, k).astype(np.float64)
            nI.append(len(I_edges))
            blocks.append(S.T.ravel())              # column-major
            dual.append(np.searchsorted(dual_edges, I_edges))
            weight.append(sign * sysd.subs[k].Dscale)
        M = torch.tensor(np.concatenate(blocks), dtype=torch.float64, device="cuda")
        dual_t = torch.tensor(np.concatenate(dual), dtype=torch.int32, device="cuda")
        w_t = torch.tensor(np.concatenate(weight), dtype=torch.float64, device="cuda")
        rng = np.random.default_rng(11)
        for call in range(2):
            nrhs = 1 + 2 * call
            x = torch.tensor(rng.standard_normal((nrhs, m)), dtype=torch.float64, device="cuda")
            y = torch.full_like(x, float("nan"))    # overwritten, never read
            ieti.ieti_interface_product_noalloc(nI, M, dual_t, w_t, x, y, m, nrhs)
            ref = torch.empty_like(x)
            ieti.ieti_apply_precond(ctx, x, ref, nrhs)
            torch.cuda.synchronize()
            err = (torch.abs(y - ref).max() / torch.abs(ref).max()).item()
            assert err < 1e-9, (call, err)
    finally:
        ieti.ieti_destroy(ctx)


def test_noalloc_product_gives_the_local_F_apply():
    """With M_k = (K_rr^-1)_II and the signs as weights the product is
    B_r K_rr^-1 B_r^T x (the oracle's W of Eq. (7)), including a subdomain
    block of size zero in the list; two calls in a row."""
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_04340_gb300 import ieti

    prob = wl.small_cases()[3]
    sysd = fd.build_system(prob)
    ctx = ieti.ieti_create(prob)
    try:
        ieti.ieti_assemble(ctx)
        ieti.ieti_factor(ctx, ieti.IETI_FP64)
        dual_edges = ieti.ieti_get_dofmap(ctx, 3)
        m = len(dual_edges)
        nI, blocks, dual, weight = [], [], [], []
        for k in range(sysd.topo.nsub):
            W = ieti.ieti_get_block(ctx, 6, k)
            I_edges = ieti.ieti_get_dofmap(ctx, 5, k)
            nI.append(len(I_edges))
            blocks.append(W.T.ravel())
            dual.append(np.searchsorted(dual_edges, I_edges))
            weight.append(ieti.ieti_get_dofmap(ctx, 7, k).astype(np.float64))
            if k == 1:
                nI.append(0)                         # an empty block between two others
        M = torch.tensor(np.concatenate(blocks), dtype=torch.float64, device="cuda")
        dual_t = torch.tensor(np.concatenate(dual), dtype=torch.int32, device="cuda")
        w_t = torch.tensor(np.concatenate(weight), dtype=torch.float64, device="cuda")
        rng = np.random.default_rng(12)
        for call in range(2):
            nrhs = 2 + call
            xh = rng.standard_normal((m, nrhs))
            x = torch.tensor(xh.T.copy(), dtype=torch.float64, device="cuda")
            y = torch.full_like(x, float("nan"))
            ieti.ieti_interface_product_noalloc(nI, M, dual_t, w_t, x, y, m, nrhs)
            torch.cuda.synchronize()
            ref = fd.apply_W(sysd, xh)
            err = np.abs(y.cpu().numpy().T - ref).max() / np.abs(ref).max()
            assert err < 1e-9, (call, err)
    finally:
        ieti.ieti_destroy(ctx)


def test_noalloc_product_rejects_oversize_request():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2501_04340_gb300 import ieti

    # 2 subdomains x 3000 interface DOFs x 1000 columns exceeds the fixed scratch:
    # rejected on the host before anything touches the device buffers
    nI = [3000, 3000]
    M = torch.zeros(1, dtype=torch.float64, device="cuda")
    dual = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(ieti.IetiError, match="INVALID_ARG"):
        ieti.ieti_interface_product_noalloc(nI, M, dual, M, M, M, 3000, 1000)
