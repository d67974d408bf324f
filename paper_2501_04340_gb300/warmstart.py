"""Learned warm start: data generation, training and evaluation through the
public API.

An instance of a WarmstartFamily has per-patch reluctivities nu and 16 source
coefficients a. The source enters the right-hand side of Eq. (3) linearly, so
the multipliers of an instance are lambda*(nu, a) = sum_c a_c Lambda_c(nu),
where Lambda_c(nu) is the solution for the unit source of coefficient c. The
network (``ieti_mlp_*``) learns only the nu dependence: input log10 nu, output
the 16 responses Lambda_c (16 m_r values); ``ieti_mlp_forward_combine`` then
forms lambda0 = sum_c a_c Lambda_c exactly. Training data come from the method
itself: one 16-load-case solve (ieti_solve with FP64 factors) per sampled nu.

The guess only changes the PCG iteration count: the stopping test
||b - F lambda|| <= tol ||b|| (Eq. (7), relative to ||b||, not to the initial
residual) is the same with or without it, and a zero guess remains the
fallback. Everything here is orchestration over the C-ABI.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import ieti
from .ieti import IETI_FP64

NCOEF = 16


@dataclasses.dataclass
class FamilySolves:
    lam: torch.Tensor        # (n, nrhs, m_r) float64, device
    iterations: np.ndarray   # PCG iterations of each solve
    relres: np.ndarray
    fields: torch.Tensor | None = None   # (n, nedge) float64 for single-load solves


def basis_context(fam):
    """Context on the family's mesh with the 16 unit sources as load cases."""
    return ieti.ieti_create(fam.base.with_params(source_params=fam.basis_source_params(), nrhs=NCOEF))


def instance_context(fam):
    """Context on the family's mesh with one load case."""
    return ieti.ieti_create(fam.base)


def solve_basis(ctx16, fam, idx, tol=1e-10, prec=IETI_FP64, maxit=2000):
    """Lambda_c(nu_i) for every i in idx: (len(idx), 16, m_r)."""
    sz = ieti.ieti_query(ctx16)
    lam = torch.zeros((len(idx), NCOEF, sz["m_r"]), dtype=torch.float64, device="cuda")
    a = torch.zeros((NCOEF, sz["nedge"]), dtype=torch.float64, device="cuda")
    its, rr = [], []
    for j, i in enumerate(idx):
        ieti.ieti_set_params(ctx16, nu=fam.nu(i))
        ieti.ieti_assemble(ctx16)
        ieti.ieti_factor(ctx16, prec)
        info = ieti.ieti_solve(ctx16, a, tol=tol, maxit=maxit, lam_out=lam[j])
        its.append(info.iterations)
        rr.append(info.relres)
    return FamilySolves(lam=lam, iterations=np.array(its), relres=np.array(rr))


def solve_instances(ctx1, fam, idx, tol=1e-8, prec=IETI_FP64, lam0=None, maxit=2000, keep_fields=False):
    """Solves instances idx one after another (lam0: (len(idx), m_r) float64
    device rows, or None for the zero guess)."""
    sz = ieti.ieti_query(ctx1)
    lam = torch.zeros((len(idx), 1, sz["m_r"]), dtype=torch.float64, device="cuda")
    fields = torch.zeros((len(idx), sz["nedge"]), dtype=torch.float64, device="cuda") if keep_fields else None
    a = torch.zeros((1, sz["nedge"]), dtype=torch.float64, device="cuda")
    its, rr = [], []
    for j, i in enumerate(idx):
        ieti.ieti_set_params(ctx1, nu=fam.nu(i), source_params=fam.source_params(i))
        ieti.ieti_assemble(ctx1)
        ieti.ieti_factor(ctx1, prec)
        info = ieti.ieti_solve(ctx1, a, lam0=None if lam0 is None else lam0[j:j + 1], tol=tol, maxit=maxit,
                               lam_out=lam[j])
        if keep_fields:
            fields[j] = a[0]
        its.append(info.iterations)
        rr.append(info.relres)
    return FamilySolves(lam=lam, iterations=np.array(its), relres=np.array(rr), fields=fields)


def he_uniform(n_in, hidden, n_out, seed):
    """Initial parameters W1|b1|W2|b2|W3|b3: W ~ U(-sqrt(6/fan_in), +), b = 0."""
    rng = np.random.default_rng(seed)
    out = []
    for (o, i) in ((hidden, n_in), (hidden, hidden), (n_out, hidden)):
        lim = np.sqrt(6.0 / i)
        out.append(rng.uniform(-lim, lim, size=(o, i)).ravel())
        out.append(np.zeros(o))
    return np.concatenate(out).astype(np.float32)


def inputs(fam, idx):
    return torch.tensor(fam.log_nu[idx], dtype=torch.float32, device="cuda").contiguous()


def train(fam, idx, basis, hidden=256, batch=64, epochs=300, lr=1e-3, decay=0.995, seed=0):
    """Network log10 nu -> (Lambda_1 .. Lambda_16) trained on the basis solves of
    the instances idx. Returns (handle, last-epoch loss in normalised units)."""
    X = inputs(fam, idx)
    T = basis.lam.reshape(len(idx), -1).to(torch.float32).contiguous()
    m = ieti.ieti_mlp_create(X.shape[1], hidden, T.shape[1], batch)
    try:
        ieti.ieti_mlp_set_params(m, he_uniform(X.shape[1], hidden, T.shape[1], seed))
        loss = ieti.ieti_mlp_fit(m, X, T, batch, epochs, lr, decay=decay, seed=seed, normalise=True)
    except Exception:
        ieti.ieti_mlp_destroy(m)
        raise
    return m, loss


def predict(m, fam, idx):
    """lambda0 rows (len(idx), m_r) float64 on the device."""
    q = ieti.ieti_mlp_query(m)
    X = inputs(fam, idx)
    coef = torch.tensor(fam.coef[idx], dtype=torch.float64, device="cuda").contiguous()
    out = torch.empty((len(idx), q["n_out"] // NCOEF), dtype=torch.float64, device="cuda")
    b = q["max_batch"]
    for s in range(0, len(idx), b):
        ieti.ieti_mlp_forward_combine(m, X[s:s + b].contiguous(), coef[s:s + b].contiguous(), out[s:s + b])
    return out
