"""Reference-element basis of the spectral element space (Sec. 2.2) and mesh
helpers for the oracle (test infrastructure only).

Legendre polynomials by the three-term recurrence of Sec. 2.2; the modal
("bubble") functions psi_p = L_{p-1} - L_{p+1} of eq. (RefBasis); the nodal
hat functions; the degree-of-freedom ordering of X in Sec. 2.2 (all bubbles
element by element, then the N-1 interior hats).

Local basis of one element, in this order:
    0: left hat  (1 - xi)/2      1: right hat (1 + xi)/2
    1+p: psi_p(xi),  p = 1..P-1
"""
from __future__ import annotations

import numpy as np


def legendre_all(pmax: int, x):
    """L_0..L_pmax at x by the recurrence of Sec. 2.2; shape (pmax+1, *x.shape)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty((pmax + 1,) + x.shape)
    out[0] = 1.0
    if pmax >= 1:
        out[1] = x
    for p in range(1, pmax):
        out[p + 1] = ((2 * p + 1) * x * out[p] - p * out[p - 1]) / (p + 1)
    return out


def legendre_deriv_all(pmax: int, x):
    """L_0'..L_pmax' at x, from the derivative of the same recurrence."""
    x = np.asarray(x, dtype=np.float64)
    L = legendre_all(pmax, x)
    d = np.zeros_like(L)
    if pmax >= 1:
        d[1] = 1.0
    for p in range(1, pmax):
        d[p + 1] = ((2 * p + 1) * (L[p] + x * d[p]) - p * d[p - 1]) / (p + 1)
    return d


def local_values(P: int, xi):
    """Local basis values (P+1 functions) at reference points xi."""
    xi = np.asarray(xi, dtype=np.float64)
    L = legendre_all(P, xi)
    out = np.empty((P + 1,) + xi.shape)
    out[0] = 0.5 * (1.0 - xi)
    out[1] = 0.5 * (1.0 + xi)
    for p in range(1, P):
        out[1 + p] = L[p - 1] - L[p + 1]
    return out


def local_derivs(P: int, xi):
    """d/dxi of the local basis (P+1 functions) at reference points xi."""
    xi = np.asarray(xi, dtype=np.float64)
    dL = legendre_deriv_all(P, xi)
    out = np.empty((P + 1,) + xi.shape)
    out[0] = -0.5
    out[1] = 0.5
    for p in range(1, P):
        out[1 + p] = dL[p - 1] - dL[p + 1]
    return out


class Mesh:
    """Partition a = x_0 < ... < x_N = b of eq. (Partition), held as element
    lengths h_i plus, for every node, its distance to a and to b (prefix and
    suffix sums).  Distances between points are always formed from whichever
    representation is smaller, so meshes refined to 2^-129 next to b stay
    exact.  Elements are 0-based here: element e spans [x_e, x_{e+1}]."""

    def __init__(self, h, a: float = 0.0, b: float | None = None):
        h = np.asarray(h, dtype=np.float64).copy()
        if h.ndim != 1 or len(h) < 1 or np.any(h <= 0):
            raise ValueError("need N >= 1 positive element lengths")
        self.h = h
        self.N = len(h)
        self.a = float(a)
        self.b = float(a + h.sum()) if b is None else float(b)
        self.dl = np.concatenate([[0.0], np.cumsum(h)])           # x_j - a
        self.dr = np.concatenate([np.cumsum(h[::-1])[::-1], [0.0]])  # b - x_j

    def gap(self, f: int, e: int) -> float:
        """x_e - x_{f+1} >= 0 for elements f < e (length strictly between)."""
        if e == f + 1:
            return 0.0
        if self.dl[e] <= self.dr[f + 1]:
            return float(self.dl[e] - self.dl[f + 1])
        return float(self.dr[f + 1] - self.dr[e])

    def node_diff(self, i: int, j: int) -> float:
        """x_i - x_j for node indices i >= j."""
        if self.dl[i] <= self.dr[j]:
            return float(self.dl[i] - self.dl[j])
        return float(self.dr[j] - self.dr[i])

    def mirrored(self) -> "Mesh":
        """The mesh reflected by x -> a + b - x (element order reversed)."""
        return Mesh(self.h[::-1], self.a, self.b)


def n_dof(N: int, P: int) -> int:
    """N_d = sum_i P_i - 1 with P_i = P (end of Sec. 2.2)."""
    return N * P - 1


def global_index(N: int, P: int):
    """Map (element e, local function k) -> index in the "full" vector.

    The full vector is X of Sec. 2.2 (bubbles element by element, then the
    interior hats) followed by the two boundary hats: node 0 at N_d and node N
    at N_d + 1.  Returns an int array idx[e, k] of shape (N, P+1).
    """
    Nd = n_dof(N, P)
    idx = np.empty((N, P + 1), dtype=np.int64)
    for e in range(N):
        left, right = e, e + 1          # node numbers
        idx[e, 0] = Nd if left == 0 else N * (P - 1) + left - 1
        idx[e, 1] = Nd + 1 if right == N else N * (P - 1) + right - 1
        for p in range(1, P):
            idx[e, 1 + p] = e * (P - 1) + p - 1
    return idx
