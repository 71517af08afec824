"""Pins for the oracle's Gauss rules: exact moments against Beta-function
closed forms (not against the rules themselves)."""
import math

import numpy as np
import pytest

from oracle.quadrature import gauss_jacobi, gauss_legendre, gl_interval


def beta(x, y):
    return math.gamma(x) * math.gamma(y) / math.gamma(x + y)


@pytest.mark.parametrize("n", [1, 2, 5, 12, 30])
def test_gauss_legendre_monomials(n):
    x, w = gauss_legendre(n)
    for k in range(2 * n):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.sum(w * x ** k) - exact) < 1e-14 * max(1.0, abs(exact)) + 1e-15


@pytest.mark.parametrize("a,b", [(0.0, 0.5), (-0.5, 0.0), (0.3, 0.7), (-0.9, 0.95), (1 - 1.3, 0), (0, 2 - 1.8)])
@pytest.mark.parametrize("n", [1, 3, 8, 16])
def test_gauss_jacobi_moments(a, b, n):
    # int (1-x)^a (1+x)^(b+k) = 2^(a+b+k+1) B(a+1, b+k+1), exact for k <= 2n-1
    x, w = gauss_jacobi(n, a, b)
    for k in range(2 * n):
        exact = 2.0 ** (a + b + k + 1) * beta(a + 1, b + k + 1)
        got = np.sum(w * (1 + x) ** k)
        assert abs(got - exact) < 2e-14 * exact


def test_gauss_jacobi_nodes_inside():
    x, w = gauss_jacobi(20, -0.6, 0.4)
    assert np.all(np.abs(x) < 1) and np.all(w > 0)


def test_gl_interval():
    x, w = gl_interval(6, 2.0, 5.0)
    assert abs(np.sum(w * x ** 3) - (5 ** 4 - 2 ** 4) / 4) < 1e-12
