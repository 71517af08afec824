"""Dense assembly of the SEM system A X = (rho M + S) X = G of eq. (lsys)
for the oracle (test infrastructure only).

Stiffness (Sec. 2.2, with the integral form used in Sec. 3.2):
    S_l[i, j] = gamma0 * int phi_i'(t) int_{s < t} (t - s)^(1-alpha) phi_j'(s) ds dt,
    gamma0 = 1 / Gamma(2 - alpha),   S = theta S_l + (1 - theta) S_r,
where S_r is the right-sided operator (kernel (s - t)^(1-alpha) over s > t).
S_r is assembled here from its own definition (by reflecting the mesh, see
`stiffness_right`), not as the transpose of S_l, so that S_r = S_l^T is a
check rather than an assumption.

The paper does not say how the singular integrals are evaluated.  The oracle
integrates every element pair (test element e, trial element f <= e) with:
  * f == e  : inner Gauss-Jacobi in the collapsed variable with weight
              (1 - tau)^(1-alpha), outer Gauss-Jacobi with weight
              (1 + xi)^(2-alpha); exact for the polynomial basis.
  * f == e-1: the common corner is the singularity; the rectangle is split
              along its diagonal and each triangle mapped by a Duffy
              transform, Gauss-Jacobi (weight rho^(2-alpha)) in the radial
              variable and Gauss-Legendre in the angular one, doubled until
              converged.
  * f <= e-2: tensor Gauss-Legendre after bisecting the larger side until
              every sub-box is no larger than its distance to the kernel's
              singular line.

Everything is in FP64.  The "full" index space is X followed by the two
boundary hats (see basis.global_index); the boundary columns carry the
boundary values c1, c2 (lifting by the boundary hats).
"""
from __future__ import annotations

import math

import numpy as np

from .basis import Mesh, global_index, local_derivs, local_values, n_dof
from .quadrature import gauss_jacobi, gauss_legendre


def gamma0(alpha: float) -> float:
    """gamma0 = 1/Gamma(2-alpha) (Sec. 4.3)."""
    return 1.0 / math.gamma(2.0 - alpha)


# ----------------------------------------------------------------------------
# element-pair integrals of the local basis derivatives
#   K[a, b] = gamma0 int_{I_e} phi_a'(t) int_{I_f, s<t} (t-s)^(1-alpha) phi_b'(s)
# ----------------------------------------------------------------------------

def pair_self(h: float, P: int, alpha: float) -> np.ndarray:
    n = P + 2
    xo, wo = gauss_jacobi(n, 0.0, 2.0 - alpha)        # outer, (1+xi)^(2-alpha)
    ti, wi = gauss_jacobi(n, 1.0 - alpha, 0.0)        # inner, (1-tau)^(1-alpha)
    eta = -1.0 + 0.5 * (1.0 + xo)[:, None] * (1.0 + ti)[None, :]   # (k, j)
    dphi_eta = local_derivs(P, eta)                   # (b, k, j)
    inner = np.einsum("bkj,j->bk", dphi_eta, wi)      # int (1-tau)^(1-alpha) phi_b'(eta)
    dphi_xi = local_derivs(P, xo)                     # (a, k)
    D = 2.0 ** (alpha - 2.0) * np.einsum("ak,k,bk->ab", dphi_xi, wo, inner)
    return gamma0(alpha) * (0.5 * h) ** (1.0 - alpha) * D


def pair_touch(he: float, hf: float, P: int, alpha: float,
               tol: float = 1e-14) -> np.ndarray:
    """Test element e immediately right of trial element f (shared node).

    The angular rule is doubled until two successive results agree to tol
    (relative) or their difference stops shrinking below 1e-13 (the roundoff
    level of the sum, 1-2e-14 of the largest entry at P = 16); the radial
    Gauss-Jacobi rule is exact for the basis."""
    xr, wr = gauss_jacobi(P + 1, 0.0, 2.0 - alpha)
    rho = 0.5 * (1.0 + xr)
    cr = 2.0 ** (alpha - 3.0) * wr                    # int_0^1 rho^(2-alpha) F

    def evaluate(nw: int) -> np.ndarray:
        xw, ww = gauss_legendre(nw)
        w = 0.5 * (1.0 + xw)
        cw = 0.5 * ww
        R, W = np.meshgrid(rho, w, indexing="ij")     # (r, q)
        C = cr[:, None] * cw[None, :]
        # triangle 1: u = he*rho, v = hf*rho*w
        k1 = C * (he + hf * W) ** (1.0 - alpha)
        da = local_derivs(P, -1.0 + 2.0 * R)          # xi = -1 + 2u/he
        db = local_derivs(P, 1.0 - 2.0 * R * W)       # eta = 1 - 2v/hf
        t1 = np.einsum("arq,rq,brq->ab", da, k1, db)
        # triangle 2: v = hf*rho, u = he*rho*w
        k2 = C * (hf + he * W) ** (1.0 - alpha)
        da = local_derivs(P, -1.0 + 2.0 * R * W)
        db = local_derivs(P, 1.0 - 2.0 * R)
        t2 = np.einsum("arq,rq,brq->ab", da, k2, db)
        return 4.0 * gamma0(alpha) * (t1 + t2)

    prev = evaluate(16)
    nw = 32
    last = np.inf
    while True:
        cur = evaluate(nw)
        d = np.max(np.abs(cur - prev)) / max(np.max(np.abs(cur)), 1e-300)
        if d <= tol:
            return cur
        # the difference has stopped shrinking at the roundoff level of the sum
        if d < 1e-13 and d >= 0.5 * last:
            return cur
        if nw >= 1024:
            raise RuntimeError("touching-pair quadrature did not converge")
        last = d
        prev = cur
        nw *= 2


def _sep_box(he, hf, g, u0, u1, v0, v1, P, alpha, n, out):
    d = g + u0 + v0
    lu, lv = u1 - u0, v1 - v0
    if max(lu, lv) > d:
        if lu >= lv:
            um = 0.5 * (u0 + u1)
            _sep_box(he, hf, g, u0, um, v0, v1, P, alpha, n, out)
            _sep_box(he, hf, g, um, u1, v0, v1, P, alpha, n, out)
        else:
            vm = 0.5 * (v0 + v1)
            _sep_box(he, hf, g, u0, u1, v0, vm, P, alpha, n, out)
            _sep_box(he, hf, g, u0, u1, vm, v1, P, alpha, n, out)
        return
    x, w = gauss_legendre(n)
    u = u0 + 0.5 * lu * (1.0 + x)
    v = v0 + 0.5 * lv * (1.0 + x)
    wu, wv = 0.5 * lu * w, 0.5 * lv * w
    K = (g + u[:, None] + v[None, :]) ** (1.0 - alpha)
    da = local_derivs(P, -1.0 + 2.0 * u / he) * wu[None, :]
    db = local_derivs(P, 1.0 - 2.0 * v / hf) * wv[None, :]
    out += (2.0 / he) * (2.0 / hf) * (da @ K @ db.T)


def pair_separated(he: float, hf: float, g: float, P: int, alpha: float,
                   n: int | None = None) -> np.ndarray:
    """Test element e right of trial element f with gap g > 0 between them.

    With u = t - x_e and v = x_{f+1} - s, t - s = g + u + v."""
    if n is None:
        n = P + 12
    out = np.zeros((P + 1, P + 1))
    _sep_box(he, hf, g, 0.0, he, 0.0, hf, P, alpha, n, out)
    return gamma0(alpha) * out


def _separated_batch(he, hf, g, P, alpha, n):
    """Vectorised pair_separated for pairs with g >= max(he, hf) (no split)."""
    x, w = gauss_legendre(n)
    t = 0.5 * (1.0 + x)
    u = he[:, None] * t[None, :]                       # (p, i)
    v = hf[:, None] * t[None, :]
    K = (g[:, None, None] + u[:, :, None] + v[:, None, :]) ** (1.0 - alpha)
    A = local_derivs(P, x) * w[None, :]                # phi_a'(xi_i) w_i
    B = local_derivs(P, -x) * w[None, :]               # phi_b'(eta_j) w_j, eta = -x
    return gamma0(alpha) * np.einsum("ai,pij,bj->pab", A, K, B, optimize=True)


def stiffness_left(mesh: Mesh, P: int, alpha: float) -> np.ndarray:
    """Full (N_d+2)^2 left-sided stiffness S_l (rows: test, cols: trial)."""
    N = mesh.N
    idx = global_index(N, P)
    nf = n_dof(N, P) + 2
    S = np.zeros((nf, nf))
    h = mesh.h
    n_sep = P + 12
    for e in range(N):
        re = idx[e]
        S[np.ix_(re, re)] += pair_self(h[e], P, alpha)
        if e >= 1:
            S[np.ix_(re, idx[e - 1])] += pair_touch(h[e], h[e - 1], P, alpha)
        if e >= 2:
            fs = np.arange(e - 1)
            g = np.array([mesh.gap(f, e) for f in fs])
            easy = g >= np.maximum(h[e], h[fs])
            if np.any(easy):
                fe = fs[easy]
                Kb = _separated_batch(np.full(len(fe), h[e]), h[fe], g[easy],
                                      P, alpha, n_sep)
                rows = np.broadcast_to(re[None, :, None], Kb.shape)
                cols = np.broadcast_to(idx[fe][:, None, :], Kb.shape)
                np.add.at(S, (rows, cols), Kb)
            for f, gf in zip(fs[~easy], g[~easy]):
                S[np.ix_(re, idx[f])] += pair_separated(h[e], h[f], gf, P, alpha,
                                                        n_sep)
    return S


def mirror_map(N: int, P: int):
    """Index permutation and signs taking a basis function phi to its
    reflection R phi(x) = phi(a + b - x), expressed in the reflected mesh.

    Returns (perm, sign) over the full index space: R phi_g = sign[g] *
    phi'_{perm[g]} where phi' is the basis of Mesh.mirrored().  Hats swap
    sides; psi_p(-xi) = (-1)^(p-1) psi_p(xi) for the bubbles."""
    idx = global_index(N, P)
    nf = n_dof(N, P) + 2
    perm = np.empty(nf, dtype=np.int64)
    sign = np.empty(nf)
    for e in range(N):
        em = N - 1 - e
        perm[idx[e, 0]] = idx[em, 1]
        sign[idx[e, 0]] = 1.0
        perm[idx[e, 1]] = idx[em, 0]
        sign[idx[e, 1]] = 1.0
        for p in range(1, P):
            perm[idx[e, 1 + p]] = idx[em, 1 + p]
            sign[idx[e, 1 + p]] = (-1.0) ** (p - 1)
    return perm, sign


def stiffness_right(mesh: Mesh, P: int, alpha: float) -> np.ndarray:
    """Full right-sided stiffness
        S_r[i, j] = gamma0 int phi_i'(t) int_{s > t} (s - t)^(1-alpha) phi_j'(s).
    Under x -> a + b - x the right-sided integral becomes a left-sided one of
    the reflected functions (the two derivative sign flips cancel), so S_r is
    the left-sided stiffness of the reflected mesh, re-indexed and signed."""
    Sm = stiffness_left(mesh.mirrored(), P, alpha)
    perm, sign = mirror_map(mesh.N, P)
    return sign[:, None] * Sm[np.ix_(perm, perm)] * sign[None, :]


def mass(mesh: Mesh, P: int) -> np.ndarray:
    """Full mass matrix M[i, j] = (phi_j, phi_i) by Gauss-Legendre."""
    N = mesh.N
    idx = global_index(N, P)
    nf = n_dof(N, P) + 2
    M = np.zeros((nf, nf))
    x, w = gauss_legendre(P + 2)
    V = local_values(P, x)
    ref = (V * w[None, :]) @ V.T
    for e in range(N):
        M[np.ix_(idx[e], idx[e])] += 0.5 * mesh.h[e] * ref
    return M


def system_full(mesh: Mesh, P: int, alpha: float, theta: float,
                rho: float) -> np.ndarray:
    """A_full = rho M + theta S_l + (1 - theta) S_r over the full index space."""
    nf = n_dof(mesh.N, P) + 2
    A = np.zeros((nf, nf))
    if theta != 0.0:
        A += theta * stiffness_left(mesh, P, alpha)
    if theta != 1.0:
        A += (1.0 - theta) * stiffness_right(mesh, P, alpha)
    if rho != 0.0:
        A += rho * mass(mesh, P)
    return A
