"""Gauss quadrature rules for the oracle (test infrastructure only).

The paper does not say how the singular double integrals of Sec. 2.2 are
evaluated.  The oracle uses classical Gauss rules built by the Golub-Welsch
method: the nodes are the eigenvalues of the symmetric tridiagonal Jacobi
matrix of the three-term recurrence, the weights are mu_0 times the squared
first components of its eigenvectors.  numpy's symmetric eigensolver is the
library step.

  gauss_legendre(n)          weight 1 on [-1, 1]
  gauss_jacobi(n, a, b)      weight (1-x)^a (1+x)^b on [-1, 1],  a, b > -1
"""
from __future__ import annotations

import math
from functools import lru_cache

import numpy as np


def _golub_welsch(alpha: np.ndarray, beta: np.ndarray, mu0: float):
    # alpha: n diagonal recurrence coefficients, beta: n-1 off-diagonal squares
    n = len(alpha)
    J = np.diag(alpha)
    if n > 1:
        off = np.sqrt(beta)
        J += np.diag(off, 1) + np.diag(off, -1)
    x, V = np.linalg.eigh(J)
    w = mu0 * V[0, :] ** 2
    return x, w


@lru_cache(maxsize=None)
def gauss_jacobi(n: int, a: float, b: float):
    """n-point Gauss-Jacobi rule for the weight (1-x)^a (1+x)^b on [-1,1].

    Exact for polynomials of degree <= 2n-1 times the weight.  Returns
    read-only (nodes, weights) arrays.
    """
    if n < 1:
        raise ValueError("n >= 1")
    if a <= -1 or b <= -1:
        raise ValueError("a, b > -1")
    k = np.arange(n, dtype=np.float64)
    s = 2.0 * k + a + b
    alpha = np.empty(n)
    with np.errstate(divide="ignore", invalid="ignore"):
        alpha[:] = (b * b - a * a) / (s * (s + 2.0))
    # first coefficient written out separately: s = a + b may be 0
    alpha[0] = (b - a) / (a + b + 2.0)
    beta = np.empty(max(n - 1, 0))
    for j in range(1, n):
        sj = 2.0 * j + a + b
        beta[j - 1] = (4.0 * j * (j + a) * (j + b) * (j + a + b)
                       / (sj * sj * (sj + 1.0) * (sj - 1.0)))
    mu0 = 2.0 ** (a + b + 1.0) * math.gamma(a + 1.0) * math.gamma(b + 1.0) \
        / math.gamma(a + b + 2.0)
    x, w = _golub_welsch(alpha, beta, mu0)
    x.setflags(write=False)
    w.setflags(write=False)
    return x, w


@lru_cache(maxsize=None)
def gauss_legendre(n: int):
    """n-point Gauss-Legendre rule on [-1, 1] (Jacobi rule with a = b = 0)."""
    if n < 1:
        raise ValueError("n >= 1")
    k = np.arange(1, n, dtype=np.float64)
    beta = k * k / (4.0 * k * k - 1.0)
    x, w = _golub_welsch(np.zeros(n), beta, 2.0)
    x.setflags(write=False)
    w.setflags(write=False)
    return x, w


def gl_interval(n: int, lo: float, hi: float):
    """Gauss-Legendre nodes and weights mapped to [lo, hi]."""
    x, w = gauss_legendre(n)
    half = 0.5 * (hi - lo)
    return lo + half * (x + 1.0), half * w
