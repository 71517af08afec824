"""Dense direct solve of eq. (lsys) for the oracle (test infrastructure only).

X* = A^{-1} G is the exact discrete SEM solution.  The preconditioned Krylov
method of Sec. 4.2 converges to this same vector; only the route differs.

Steps: symmetric equilibration by powers of two (exact in binary floating
point), LU with partial pivoting (LAPACK through scipy, the library step),
then iterative refinement with the residual formed in numpy's long double.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .assemble import system_full
from .basis import Mesh, n_dof
from .load import load_frac_powers, load_legendre_ab


def equilibrate(A: np.ndarray) -> np.ndarray:
    """s_i = 2^round(-log2|A_ii| / 2), so that diag(s A s) lies in [1/2, 2]."""
    d = np.abs(np.diag(A))
    return np.exp2(np.round(-0.5 * np.log2(d)))


def dense_solve(A: np.ndarray, b: np.ndarray, refine: int = 3):
    """Solve A x = b (b may have several columns).  Returns (x, corr) where
    corr is the relative size of the last refinement correction."""
    b2 = b.reshape(len(b), -1)
    s = equilibrate(A)
    As = s[:, None] * A * s[None, :]
    bs = s[:, None] * b2
    lu = sla.lu_factor(As, check_finite=True)
    y = sla.lu_solve(lu, bs)
    Al = As.astype(np.longdouble)
    corr = np.inf
    for _ in range(refine):
        r = (bs.astype(np.longdouble) - Al @ y.astype(np.longdouble)).astype(np.float64)
        dy = sla.lu_solve(lu, r)
        y = y + dy
        corr = float(np.linalg.norm(dy) / max(np.linalg.norm(y), 1e-300))
    x = s[:, None] * y
    return x.reshape(b.shape), corr


def load_vector(mesh: Mesh, P: int, rhs) -> np.ndarray:
    """Full load vector for rhs = ("frac_powers", terms) |
    ("legendre_ab", coeffs) | ("load_vector", G over the N_d unknowns)."""
    kind, data = rhs
    if kind == "frac_powers":
        return load_frac_powers(mesh, P, data)
    if kind == "legendre_ab":
        return load_legendre_ab(mesh, P, data)
    if kind == "load_vector":
        G = np.zeros(n_dof(mesh.N, P) + 2)
        G[: n_dof(mesh.N, P)] = np.asarray(data, dtype=np.float64)
        return G
    raise ValueError(kind)


def solve_problem(mesh: Mesh, P: int, alpha: float, theta: float, rho: float,
                  c1: float, c2: float, rhs, A_full=None):
    """Exact discrete solution X* (X's ordering of Sec. 2.2).

    The boundary values enter through the two boundary hats: their columns
    move to the right-hand side.  Returns (X, info)."""
    Nd = n_dof(mesh.N, P)
    if A_full is None:
        A_full = system_full(mesh, P, alpha, theta, rho)
    G = load_vector(mesh, P, rhs)
    rhs_i = G[:Nd] - A_full[:Nd, Nd:] @ np.array([c1, c2])
    if Nd == 0:
        return np.zeros(0), {"corr": 0.0}
    X, corr = dense_solve(A_full[:Nd, :Nd], rhs_i)
    return X, {"corr": corr, "A_full": A_full, "G": G}
