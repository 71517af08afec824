"""H-matrix approximation A~ = rho M + theta H + (1 - theta) H^T of Sec. 3
for the oracle (test infrastructure only), returned as a dense matrix over the
N_d unknowns in X's ordering.

  * Clusters are element index ranges [e0, e1), split in halves until at most
    `leaf` elements remain (the paper does not say how its cluster tree is
    built).  A cluster owns the bubbles of its elements and the hats at its
    elements' right nodes (never the boundary node b).
  * The support of a cluster is the union of its functions' supports
    (Sec. 3.2): [x_e0, x_{min(e1+1, N)}].
  * Admissibility, eq. (admis): max(diam tau, diam sigma) <= lambda * dist
    (rule "max"); rule "min" admits min(diam tau, diam sigma) <= lambda *
    dist, the expansion then being taken about the smaller cluster (Remark
    after the Lemma), whose diameter over the distance is all the Lemma's
    bound (lambda/(2+lambda))^R needs.
  * Admissible block with the test cluster tau right of the trial cluster
    sigma: S_l(tau, sigma) ~ Q W^T, Q_{i,nu} = gamma0 int h_nu phi_i',
    W_{j,nu} = int g_nu phi_j' (Sec. 3.2), from the Taylor expansion
    eq. (eqn:Lexpan) about the centre s0 of sigma.  Following Remark 3.1 the
    expansion is taken in t about the centre t0 of tau instead when tau is
    the smaller cluster.  In the mirrored position S_l is zero, so
    A~(sigma, tau) = (1 - theta) (Q W^T)^T.
  * Inadmissible leaves keep the exact entries (end of Sec. 3.2).

Scaling: g_nu is written as ((s - s0)/r)^nu with r the half-length of the
expansion cluster and h_nu carries r^nu; the product is unchanged and the
factors stay in range on meshes refined to 2^-129.
"""
from __future__ import annotations

import math

import numpy as np

from .assemble import gamma0
from .basis import Mesh, global_index, local_derivs, n_dof
from .quadrature import gauss_legendre


class Cluster:
    def __init__(self, e0: int, e1: int):
        self.e0, self.e1 = e0, e1
        self.kids: list[Cluster] = []


def cluster_tree(N: int, leaf: int) -> Cluster:
    def build(e0, e1):
        c = Cluster(e0, e1)
        if e1 - e0 > leaf:
            mid = (e0 + e1) // 2
            c.kids = [build(e0, mid), build(mid, e1)]
        return c
    return build(0, N)


def support(N: int, c: Cluster):
    """Node indices (lo, hi) of the cluster's support interval."""
    return c.e0, min(c.e1 + 1, N)


def diam(mesh: Mesh, c: Cluster) -> float:
    lo, hi = support(mesh.N, c)
    return mesh.node_diff(hi, lo)


def dist(mesh: Mesh, c1: Cluster, c2: Cluster) -> float:
    l1, h1 = support(mesh.N, c1)
    l2, h2 = support(mesh.N, c2)
    if h1 < l2:
        return mesh.node_diff(l2, h1)
    if h2 < l1:
        return mesh.node_diff(l1, h2)
    return 0.0


def admissible(mesh: Mesh, t: Cluster, s: Cluster, lam: float, rule: str = "max") -> bool:
    d = dist(mesh, t, s)
    pick = max if rule == "max" else min
    return d > 0.0 and pick(diam(mesh, t), diam(mesh, s)) <= lam * d


def block_leaves(mesh: Mesh, root: Cluster, lam: float, rule: str = "max"):
    """Leaves of the block tree: list of (tau, sigma, is_admissible)."""
    out = []

    def rec(t, s):
        if admissible(mesh, t, s, lam, rule):
            out.append((t, s, True))
        elif not t.kids or not s.kids:
            out.append((t, s, False))
        else:
            for tk in t.kids:
                for sk in s.kids:
                    rec(tk, sk)
    rec(root, root)
    return out


def cluster_dofs(N: int, P: int, c: Cluster) -> np.ndarray:
    """Unknowns (X's ordering) owned by a cluster."""
    idx = global_index(N, P)
    Nd = n_dof(N, P)
    out = []
    for e in range(c.e0, c.e1):
        out.extend(idx[e, 2:].tolist())
        if e + 1 < N:
            out.append(int(idx[e, 1]))
    return np.array([i for i in out if i < Nd], dtype=np.int64)


def _taylor_coeffs(alpha: float, R: int) -> np.ndarray:
    """prod_{l=1}^{nu} (2 - alpha - l) / nu!,  nu = 0..R-1."""
    c = np.empty(R)
    c[0] = 1.0
    for nu in range(1, R):
        c[nu] = c[nu - 1] * (2.0 - alpha - nu) / nu
    return c


def _moments(mesh: Mesh, P: int, c: Cluster, func, n: int) -> np.ndarray:
    """M[i, nu] = int func_nu(x) phi_i'(x) dx for the cluster's unknowns,
    integrating element by element over the cluster's support.
    func(e, xq) -> (R, nq) values on element e at reference nodes xq."""
    N = mesh.N
    idx = global_index(N, P)
    dofs = cluster_dofs(N, P, c)
    pos = {int(d): k for k, d in enumerate(dofs)}
    x, w = gauss_legendre(n)
    dphi = local_derivs(P, x) * w[None, :]          # (k, q): w_q phi_k'(x_q)
    out = None
    lo, hi = support(N, c)
    for e in range(lo, hi):
        vals = func(e, x)                           # (R, q)
        m = dphi @ vals.T                           # (k, R): int phi' * f, (2/h)(h/2) = 1
        if out is None:
            out = np.zeros((len(dofs), vals.shape[0]))
        for k in range(P + 1):
            g = int(idx[e, k])
            if g in pos:
                out[pos[g]] += m[k]
    return out


def lowrank_factors(mesh: Mesh, P: int, alpha: float, tau: Cluster,
                    sig: Cluster, R: int, expand: str = "auto"):
    """(Q, W) with S_l(tau, sigma) ~ Q W^T, tau's support right of sigma's."""
    N = mesh.N
    lo_t, hi_t = support(N, tau)
    lo_s, hi_s = support(N, sig)
    assert hi_s < lo_t
    r_s = 0.5 * mesh.node_diff(hi_s, lo_s)
    r_t = 0.5 * mesh.node_diff(hi_t, lo_t)
    nu = np.arange(R, dtype=np.float64)
    c = _taylor_coeffs(alpha, R)
    n = P + R + 16
    if expand == "auto":
        expand = "s" if r_s <= r_t else "t"

    if expand == "s":
        # k(t,s) ~ sum_nu c_nu (-1)^nu (t-s0)^(1-alpha-nu) (s-s0)^nu
        def hfun(e, x):
            d = mesh.node_diff(e, hi_s) + 0.5 * mesh.h[e] * (1.0 + x) + r_s  # t - s0
            return ((-1.0) ** nu * c * r_s ** nu)[:, None] * d[None, :] ** (1.0 - alpha - nu[:, None])

        def gfun(f, x):
            y = (mesh.node_diff(f, lo_s) + 0.5 * mesh.h[f] * (1.0 + x) - r_s) / r_s
            return y[None, :] ** nu[:, None]
        Q = gamma0(alpha) * _moments(mesh, P, tau, hfun, n)
        W = _moments(mesh, P, sig, gfun, n)
    else:
        # k(t,s) ~ sum_nu c_nu (t0-s)^(1-alpha-nu) (t-t0)^nu
        def gfun(e, x):
            y = (mesh.node_diff(e, lo_t) + 0.5 * mesh.h[e] * (1.0 + x) - r_t) / r_t
            return y[None, :] ** nu[:, None]

        def hfun(f, x):
            d = r_t + mesh.node_diff(lo_t, f + 1) + 0.5 * mesh.h[f] * (1.0 - x)  # t0 - s
            return (c * r_t ** nu)[:, None] * d[None, :] ** (1.0 - alpha - nu[:, None])
        Q = gamma0(alpha) * _moments(mesh, P, tau, gfun, n)
        W = _moments(mesh, P, sig, hfun, n)
    return Q, W


def hmatrix_dense(mesh: Mesh, P: int, alpha: float, theta: float,
                  A_full: np.ndarray, R: int, lam: float = 1.0, leaf: int = 2,
                  expand: str = "auto", rule: str = "max"):
    """Dense A~ over the N_d unknowns, built from the exact A (A_full from
    assemble.system_full) by replacing every admissible block.  Returns
    (A_tilde, blocks) with blocks = list of (tau, sigma, admissible)."""
    N = mesh.N
    Nd = n_dof(N, P)
    At = np.array(A_full[:Nd, :Nd], copy=True)
    root = cluster_tree(N, leaf)
    blocks = block_leaves(mesh, root, lam, rule)
    for t, s, adm in blocks:
        if not adm:
            continue
        lo_t, _ = support(N, t)
        _, hi_s = support(N, s)
        if hi_s >= lo_t:             # tau left of sigma: filled from the mirror
            continue
        Q, W = lowrank_factors(mesh, P, alpha, t, s, R, expand)
        rt, rs = cluster_dofs(N, P, t), cluster_dofs(N, P, s)
        At[np.ix_(rt, rs)] = theta * (Q @ W.T)
        At[np.ix_(rs, rt)] = (1.0 - theta) * (W @ Q.T)
    return At, blocks
