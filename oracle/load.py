"""Load vector G of eq. (lsys) for the oracle (test infrastructure only).

G_i = (f, phi_i) over the full index space (X's ordering followed by the two
boundary hats).  Three ways to give f:

  frac_powers : f(x) = sum_k c_k (x - a)^mu_k  [side "a"]
                     + sum_k d_k (b - x)^nu_k  [side "b"],   exponents > -1.
                Terms with negative exponents are integrable singularities at
                an endpoint; the end element uses Gauss-Jacobi with the
                matching weight, the other elements composite Gauss-Legendre
                on pieces that double in distance from the endpoint.
  legendre_ab : f(x) = sum_k g_k L_k(xi_[a,b](x)), a polynomial.
  load_vector : G given directly.
"""
from __future__ import annotations

import numpy as np

from .basis import Mesh, global_index, legendre_all, local_values, n_dof
from .quadrature import gauss_jacobi, gauss_legendre


def _power_moments_end(h: float, mu: float, P: int, at_left: bool) -> np.ndarray:
    """int over the end element of dist^mu * phi_k, dist measured from the
    endpoint the element touches."""
    x, w = gauss_jacobi(P + 2, 0.0 if at_left else mu, mu if at_left else 0.0)
    V = local_values(P, x)
    return (0.5 * h) ** (1.0 + mu) * (V @ w)


def _power_moments_inner(d0: float, h: float, mu: float, P: int,
                         at_left: bool, n: int) -> np.ndarray:
    """int over an element at distance d0 > 0 from the endpoint of
    dist^mu * phi_k; pieces [c, 2c] keep every piece as long as its distance."""
    x, w = gauss_legendre(n)
    acc = np.zeros(P + 1)
    lo = 0.0                         # offset from the element's near node
    while lo < h:
        hi = min(h, lo + (d0 + lo))
        off = lo + 0.5 * (hi - lo) * (1.0 + x)     # offsets in [lo, hi]
        wt = 0.5 * (hi - lo) * w
        val = (d0 + off) ** mu
        # reference coordinate, measured from the node nearest the endpoint
        xi = -1.0 + 2.0 * off / h if at_left else 1.0 - 2.0 * off / h
        acc += local_values(P, xi) @ (wt * val)
        lo = hi
    return acc


def load_frac_powers(mesh: Mesh, P: int, terms) -> np.ndarray:
    """terms: iterable of (coef, exponent, side) with side in {"a", "b"}."""
    N = mesh.N
    idx = global_index(N, P)
    G = np.zeros(n_dof(N, P) + 2)
    n = P + 24
    for coef, mu, side in terms:
        if mu <= -1.0:
            raise ValueError("exponent must exceed -1")
        for e in range(N):
            if side == "a":
                d0 = mesh.dl[e]
                m = (_power_moments_end(mesh.h[e], mu, P, True) if e == 0
                     else _power_moments_inner(d0, mesh.h[e], mu, P, True, n))
            elif side == "b":
                d0 = mesh.dr[e + 1]
                m = (_power_moments_end(mesh.h[e], mu, P, False) if e == N - 1
                     else _power_moments_inner(d0, mesh.h[e], mu, P, False, n))
            else:
                raise ValueError("side must be 'a' or 'b'")
            np.add.at(G, idx[e], coef * m)
    return G


def load_legendre_ab(mesh: Mesh, P: int, coeffs) -> np.ndarray:
    """f = sum_k g_k L_k(xi_[a,b](x)) against the local basis (Sec. 2.2 load
    vector): f phi has degree K + P on every element, so the n-point
    Gauss-Legendre rule with 2n - 1 >= K + P, n = (K + P) // 2 + 1, is exact."""
    coeffs = np.asarray(coeffs, dtype=np.float64)
    K = len(coeffs) - 1
    N = mesh.N
    idx = global_index(N, P)
    G = np.zeros(n_dof(N, P) + 2)
    x, w = gauss_legendre((K + P) // 2 + 1)
    V = local_values(P, x)
    L = mesh.b - mesh.a
    for e in range(N):
        y = mesh.dl[e] + 0.5 * mesh.h[e] * (1.0 + x)   # x - a
        f = coeffs @ legendre_all(K, -1.0 + 2.0 * y / L)
        np.add.at(G, idx[e], 0.5 * mesh.h[e] * (V @ (w * f)))
    return G
