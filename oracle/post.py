"""Flux density B = curl a and the error eps_B of Sec. 3 (oracle, test
infrastructure).

eps_B = sqrt(sum_k ||B_ana - B_num||^2_{L2(Omega^(k))}) (Sec. 3), evaluated by
Gauss quadrature with ``nq`` points per direction per knot span.
"""
from __future__ import annotations

import numpy as np

from . import discretise as dz


def sine_B(X, amp=1.0):
    """curl of A = amp (sin(pi y) sin(pi z), sin(pi x) sin(pi z), sin(pi x) sin(pi y))."""
    x, y, z = X[..., 0], X[..., 1], X[..., 2]
    pi = np.pi
    return amp * pi * np.stack([np.sin(pi * x) * (np.cos(pi * y) - np.cos(pi * z)),
                                np.sin(pi * y) * (np.cos(pi * z) - np.cos(pi * x)),
                                np.sin(pi * z) * (np.cos(pi * x) - np.cos(pi * y))], -1)


def flux_l2(prob, mesh, a, B_exact=None, nq=None, rhs=0, patches=None):
    """Returns (||B_num||_L2, ||B_exact - B_num||_L2) for load case ``rhs``;
    B_num = DF curl_hat(a) / det DF at the quadrature points. ``patches``
    restricts both norms to those patches (default: the whole domain)."""
    nb2 = 0.0
    err2 = 0.0
    for q in (range(prob.npatch_total) if patches is None else patches):
        for gids, val, curl, X, DF, wts in dz._patch_element_loop(prob, mesh, q, nq=nq):
            det = np.linalg.det(DF)
            ch = np.einsum("iqa,i->qa", curl, a[gids, rhs])
            B = np.einsum("qra,qa->qr", DF, ch) / det[:, None]
            w = wts * np.abs(det)
            nb2 += np.sum(w * np.sum(B * B, -1))
            if B_exact is not None:
                Be = B_exact(X)
                err2 += np.sum(w * np.sum((Be - B) ** 2, -1))
    return np.sqrt(nb2), np.sqrt(err2)
