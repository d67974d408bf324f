"""B-spline bases of the curl-conforming spline space (oracle, test infrastructure).

Sec. 2 (discrete space W of Eq. (3)): the paper uses the curl-conforming IGA
multipatch space of its reference [Mally 2024] / Buffa et al. and states that the
DOFs correspond to edges of the (control) mesh (Sec. 2.2, tree-cotree paragraph).

Reading: "degree p" is the degree of the H1 spline space. The edge space's
component d has degree p-1 in direction d and p in the others; its 1D basis is
the Curry-Schoenberg scaled D_i = p / (t_{i+p+1} - t_{i+1}) N_{i+1,p-1}, so that
N_{i,p}' = D_{i-1} - D_i and the gradient of the H1 basis is the control-mesh
node-edge incidence matrix.
"""
from __future__ import annotations

import numpy as np


def open_uniform_knots(p: int, nspan: int) -> np.ndarray:
    """Open uniform knot vector on [0, 1]: p+1 repeated end knots, single inner
    knots (maximal smoothness C^{p-1} inside a patch)."""
    inner = [i / nspan for i in range(1, nspan)]
    return np.array([0.0] * (p + 1) + inner + [1.0] * (p + 1))


def bspline_all(t: np.ndarray, q: int, x: float) -> np.ndarray:
    """Values of all B-splines N_{i,q}, i = 0 .. len(t)-q-2, at x by the Cox-de
    Boor recursion written out level by level (plain loops).

    Half-open spans [t_i, t_{i+1}); x must lie strictly inside (0, 1) or on an
    inner knot (the quadrature points used here always do)."""
    m = len(t) - 1
    N = np.zeros(m)
    for i in range(m):
        if t[i] <= x < t[i + 1]:
            N[i] = 1.0
    for d in range(1, q + 1):
        Nn = np.zeros(m - d)
        for i in range(m - d):
            v = 0.0
            den1 = t[i + d] - t[i]
            if den1 > 0:
                v += (x - t[i]) / den1 * N[i]
            den2 = t[i + d + 1] - t[i + 1]
            if den2 > 0:
                v += (t[i + d + 1] - x) / den2 * N[i + 1]
            Nn[i] = v
        N = Nn
    return N


def h1_values(t: np.ndarray, p: int, x: float) -> np.ndarray:
    """N_{i,p}(x) for i = 0 .. n+p-1."""
    return bspline_all(t, p, x)


def edge_values(t: np.ndarray, p: int, x: float) -> np.ndarray:
    """D_i(x) = p / (t_{i+p+1} - t_{i+1}) N_{i+1,p-1}(x) for i = 0 .. n+p-2."""
    Nm = bspline_all(t, p - 1, x)
    n = len(t) - p - 1
    D = np.zeros(n - 1)
    for i in range(n - 1):
        den = t[i + p + 1] - t[i + 1]
        D[i] = p / den * Nm[i + 1] if den > 0 else 0.0
    return D


def h1_derivs(t: np.ndarray, p: int, x: float) -> np.ndarray:
    """N_{i,p}'(x) by the textbook derivative formula
    N' = p/(t_{i+p}-t_i) N_{i,p-1} - p/(t_{i+p+1}-t_{i+1}) N_{i+1,p-1}."""
    Nm = bspline_all(t, p - 1, x)
    n = len(t) - p - 1
    dN = np.zeros(n)
    for i in range(n):
        v = 0.0
        den1 = t[i + p] - t[i]
        if den1 > 0:
            v += p / den1 * Nm[i]
        den2 = t[i + p + 1] - t[i + 1]
        if den2 > 0:
            v -= p / den2 * Nm[i + 1]
        dN[i] = v
    return dN


def gauss_legendre(nq: int):
    """Gauss-Legendre points and weights on [0, 1]."""
    x, w = np.polynomial.legendre.leggauss(nq)
    return 0.5 * (x + 1.0), 0.5 * w
