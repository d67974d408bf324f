"""Pins of the oracle's 1D bases (Sec. 2 discrete space; Curry-Schoenberg edge basis)."""
import numpy as np
import pytest
from scipy.interpolate import BSpline

from oracle import splines


@pytest.mark.parametrize("p", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [1, 2, 5])
def test_bspline_values_match_scipy(p, n):
    t = splines.open_uniform_knots(p, n)
    xs = np.random.default_rng(p * 10 + n).uniform(0, 1, 17)
    ref = BSpline.design_matrix(xs, t, p).toarray()     # library routine
    mine = np.array([splines.h1_values(t, p, x) for x in xs])
    np.testing.assert_allclose(mine, ref, atol=1e-14)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_partition_of_unity_and_edge_normalisation(p):
    n = 4
    t = splines.open_uniform_knots(p, n)
    for x in np.linspace(0.01, 0.99, 23):
        assert abs(splines.h1_values(t, p, x).sum() - 1.0) < 1e-14
    # Curry-Schoenberg: every D_i integrates to one (closed form)
    xq, wq = splines.gauss_legendre(p + 1)
    integ = np.zeros(n + p - 1)
    for s in range(n):
        for x, w in zip(xq, wq):
            integ += w / n * splines.edge_values(t, p, (s + x) / n)
    np.testing.assert_allclose(integ, 1.0, atol=1e-13)


@pytest.mark.parametrize("p", [1, 2, 3])
def test_derivative_is_difference_of_edge_functions(p):
    """N_i' = D_{i-1} - D_i: the gradient of the H1 basis is the incidence matrix."""
    n = 3
    t = splines.open_uniform_knots(p, n)
    for x in np.linspace(0.013, 0.987, 19):
        dN = splines.h1_derivs(t, p, x)
        D = splines.edge_values(t, p, x)
        Dp = np.concatenate([[0.0], D, [0.0]])
        np.testing.assert_allclose(dN, Dp[:-1] - Dp[1:], atol=1e-12)
        # independent check by central differences of the values
        h = 1e-6
        fd = (splines.h1_values(t, p, x + h) - splines.h1_values(t, p, x - h)) / (2 * h)
        np.testing.assert_allclose(dN, fd, atol=1e-6 * max(1, p * n))


def test_gauss_legendre_exactness():
    for nq in range(1, 6):
        x, w = splines.gauss_legendre(nq)
        for k in range(2 * nq):
            assert abs(np.sum(w * x ** k) - 1.0 / (k + 1)) < 1e-14
