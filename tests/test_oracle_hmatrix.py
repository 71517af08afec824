"""Pins for the oracle's H-matrix approximation (Sec. 3): the block tree
partitions the matrix, the Lemma's kernel error bound, Theorem 2's entry
bounds, the exponential decay of ||A - A~||_F in R (Fig. matrixerror), and
A~ -> A as R grows."""
import math

import numpy as np
import pytest

from oracle.assemble import system_full
from oracle.basis import Mesh, global_index, n_dof
from oracle.hmatrix import (_taylor_coeffs, block_leaves, cluster_dofs,
                            cluster_tree, hmatrix_dense, support)
from paper_1808_02937_gb300 import workloads as W


@pytest.fixture(scope="module")
def graded():
    N, P, alpha = 40, 3, 1.6
    mesh = Mesh(W.mesh_graded(N, 5.0, 0.0, 10.0), 0.0, 10.0)
    A = system_full(mesh, P, alpha, 1.0, 0.0)
    return mesh, P, alpha, A


def test_block_tree_partitions_matrix(graded):
    mesh, P, alpha, A = graded
    N = mesh.N
    Nd = n_dof(N, P)
    cover = np.zeros((Nd, Nd), dtype=int)
    for t, s, adm in block_leaves(mesh, cluster_tree(N, 2), 1.0):
        cover[np.ix_(cluster_dofs(N, P, t), cluster_dofs(N, P, s))] += 1
    assert np.all(cover == 1)


def test_lemma_kernel_error_bound():
    # |k - k~| <= (1 + lam/2) (lam/(2+lam))^R / (a' - d')^(alpha-1)  (eq. (eqn:errkernel))
    rng = np.random.default_rng(1)
    alpha = 1.37
    for lam in (1.0, 0.5, 0.25):
        for _ in range(20):
            c = rng.uniform(0, 1)
            dsig = rng.uniform(0.1, 1.0)
            d_ = c + dsig
            dist = max(dsig, rng.uniform(0.1, 1.0)) / lam
            a_ = d_ + dist
            b_ = a_ + rng.uniform(0.05, lam * dist)
            s0 = 0.5 * (c + d_)
            for R in (1, 3, 6, 10):
                cf = _taylor_coeffs(alpha, R)
                t = rng.uniform(a_, b_, 7)
                s = rng.uniform(c, d_, 7)
                nu = np.arange(R)
                kt = np.sum(((-1.0) ** nu * cf)[None, :] * (t - s0)[:, None] ** (1 - alpha - nu)
                            * (s - s0)[:, None] ** nu, axis=1)
                err = np.abs((t - s) ** (1 - alpha) - kt)
                bound = (1 + lam / 2) * (lam / (2 + lam)) ** R / (a_ - d_) ** (alpha - 1)
                assert np.all(err <= bound * (1 + 1e-12))


def test_theorem2_entry_bounds(graded):
    mesh, P, alpha, A = graded
    N = mesh.N
    Nd = n_dof(N, P)
    lam, R = 1.0, 3
    At, blocks = hmatrix_dense(mesh, P, alpha, 1.0, A, R, lam, leaf=2, expand="s")
    idx = global_index(N, P)
    elem_of = {}
    for e in range(N):
        for k in range(2, P + 1):
            elem_of[int(idx[e, k])] = ("bubble", e)
        if e + 1 < N:
            elem_of[int(idx[e, 1])] = ("hat", e)
    delta = lam / (2 + lam)
    g = math.gamma(2 - alpha)
    checked = 0
    for t, s, adm in blocks:
        if not adm:
            continue
        lo_t, hi_t = support(N, t)
        lo_s, hi_s = support(N, s)
        if hi_s >= lo_t:
            continue
        ad = mesh.node_diff(lo_t, hi_s)              # a' - d'
        ds0 = 0.5 * mesh.node_diff(hi_s, lo_s)       # d' - s0
        c0 = (1 + lam / 2) * (R + 1 + lam / 2) / (ad + ds0) ** alpha
        for i in cluster_dofs(N, P, t):
            kind_i, e = elem_of[int(i)]
            hi_ = mesh.h[e]
            for j in cluster_dofs(N, P, s):
                kind_j, _ = elem_of[int(j)]
                err = abs(A[i, j] - At[i, j])
                if kind_i == "bubble" and kind_j == "bubble":
                    bound = 8 * hi_ * c0 / g * delta ** R
                elif kind_i == "bubble":
                    bound = 4 * hi_ * c0 / g * delta ** R
                else:
                    hn = mesh.h[e + 1]
                    bound = 2 * (hi_ + hn) * c0 / g * delta ** R
                assert err <= bound, (kind_i, kind_j, err, bound)
                checked += 1
    assert checked > 100


@pytest.mark.parametrize("lam", [1.0, 0.5, 0.25])
def test_frobenius_error_decays_exponentially(graded, lam):
    # leaf clusters of one element, so that every lam has admissible blocks
    mesh, P, alpha, A = graded
    Nd = n_dof(mesh.N, P)
    errs = []
    for R in (2, 4, 6, 8):
        At, blocks = hmatrix_dense(mesh, P, alpha, 1.0, A, R, lam, leaf=1)
        assert any(b[2] for b in blocks)
        errs.append(np.linalg.norm(A[:Nd, :Nd] - At))
    rates = [errs[k + 1] / errs[k] for k in range(3)]
    # (lam/(2+lam))^2 per two ranks: 1/9 at lam = 1
    assert all(r < 2.0 * (lam / (2 + lam)) ** 2 for r in rates), rates


def test_large_rank_recovers_exact_matrix(graded):
    mesh, P, alpha, A = graded
    Nd = n_dof(mesh.N, P)
    for expand in ("s", "t", "auto"):
        At, _ = hmatrix_dense(mesh, P, alpha, 0.6, system_full(mesh, P, alpha, 0.6, 0.3),
                              28, 1.0, leaf=2, expand=expand)
        A2 = system_full(mesh, P, alpha, 0.6, 0.3)[:Nd, :Nd]
        assert np.abs(At - A2).max() < 1e-13 * np.abs(A2).max()


# ---- the "min" admissibility on a geometrically graded mesh ----------------
@pytest.fixture(scope="module")
def geometric():
    N, P, alpha = 36, 3, 1.45
    mesh = Mesh(W.mesh_geometric_two_sided(N, 0.45), 0.0, 1.0)
    A = system_full(mesh, P, alpha, 0.7, 0.4)
    return mesh, P, alpha, A


def test_min_rule_admits_more_and_partitions(geometric):
    mesh, P, alpha, A = geometric
    N = mesh.N
    Nd = n_dof(N, P)
    root = cluster_tree(N, 2)
    bmax = block_leaves(mesh, root, 1.0, "max")
    bmin = block_leaves(mesh, root, 1.0, "min")
    cover = np.zeros((Nd, Nd), dtype=int)
    for t, s, adm in bmin:
        cover[np.ix_(cluster_dofs(N, P, t), cluster_dofs(N, P, s))] += 1
    assert np.all(cover == 1)

    def dense_entries(bl):
        return sum(len(cluster_dofs(N, P, t)) * len(cluster_dofs(N, P, s))
                   for t, s, adm in bl if not adm)
    assert dense_entries(bmin) < 0.5 * dense_entries(bmax)


@pytest.mark.parametrize("expand", ["auto", "s_always"])
def test_min_rule_converges_only_about_the_smaller_cluster(geometric, expand):
    # with min(diam) <= lambda dist only the smaller cluster's expansion is
    # covered by the Lemma: about it the error decays like (1/3)^R; expanding
    # about the trial cluster regardless (a plausible mistake) does not
    mesh, P, alpha, A = geometric
    Nd = n_dof(mesh.N, P)
    ex = "auto" if expand == "auto" else "s"
    errs = []
    for R in (4, 8, 12):
        At, blocks = hmatrix_dense(mesh, P, alpha, 0.7, A, R, 1.0, leaf=2, expand=ex, rule="min")
        errs.append(np.abs(A[:Nd, :Nd] - At).max())
    if expand == "auto":
        assert errs[1] < 0.05 * errs[0] and errs[2] < 0.05 * errs[1], errs
    else:
        assert not (errs[1] < 0.05 * errs[0] and errs[2] < 0.05 * errs[1]), errs


def test_min_rule_large_rank_recovers_exact_matrix(geometric):
    mesh, P, alpha, A = geometric
    Nd = n_dof(mesh.N, P)
    At, _ = hmatrix_dense(mesh, P, alpha, 0.7, A, 30, 1.0, leaf=2, rule="min")
    assert np.abs(At - A[:Nd, :Nd]).max() < 1e-13 * np.abs(A[:Nd, :Nd]).max()
