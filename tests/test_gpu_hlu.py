"""GPU parity of the H-matrix approximation, the H-LU factorisation and the
H-triangular solves (Sec. 3, Sec. 4.1) against the oracle, through the C ABI."""
import numpy as np
import pytest

from oracle.assemble import system_full
from oracle.basis import Mesh, n_dof
from oracle.hmatrix import hmatrix_dense
from oracle.load import load_frac_powers
from oracle.solve import dense_solve, solve_problem
from paper_1808_02937_gb300 import hfsem as H
from paper_1808_02937_gb300 import workloads as W
from tests._common import ensure_built, rel_err

pytestmark = pytest.mark.gpu

CASES = [
    # name, h, a, b, P, alpha, theta, rho, leaf, R
    ("uniform", W.mesh_uniform(24), 0.0, 1.0, 3, 1.5, 0.5, 0.0, 2, 4),
    ("graded5", W.mesh_graded(20, 5.0, 0.0, 10.0), 0.0, 10.0, 3, 1.6, 1.0, 0.0, 1, 5),
    ("geo2", W.mesh_geometric_two_sided(16, 0.5), 0.0, 1.0, 4, 1.3, 0.7, 1.0, 1, 6),
    ("ragged-theta0", W.mesh_graded(19, 2.0), 0.0, 1.0, 2, 1.8, 0.0, 0.4, 2, 3),
]


@pytest.fixture(scope="module")
def lib():
    return ensure_built()


@pytest.mark.parametrize("rule", ["max", "min"])
@pytest.mark.parametrize("prec", [H.PREC_FP64, H.PREC_MIXED])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_hmatrix_entries_match_oracle(lib, case, prec, rule):
    name, h, a, b, P, alpha, theta, rho, leaf, R = case
    sys = H.hfsem_assemble([H.make_problem(h, P, alpha, theta, rho, a=a, b=b, matvec=1)])
    adm = H.ADM_MAX if rule == "max" else H.ADM_MIN
    fac = H.hfsem_hlu_factor(sys, H.hopts(R=R, lam=1.0, tol_hlu=0.0, precision=prec,
                                          leaf_elems=leaf, build_only=1, admissibility=adm))
    At_gpu = H.hfsem_hmatrix_dense(fac, 0)
    m = Mesh(h, a, b)
    At, _ = hmatrix_dense(m, P, alpha, theta, system_full(m, P, alpha, theta, rho), R, 1.0, leaf,
                          rule=rule)
    tol = 1e-12 if prec == H.PREC_FP64 else 2e-6
    assert np.abs(At_gpu - At).max() <= tol * np.abs(At).max()


@pytest.mark.parametrize("rule", ["max", "min"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_hlu_exact_at_zero_tolerance(lib, case, rule):
    # Tol_HLU = 0 and no rank cap: H-LU is an exact LU of A~
    name, h, a, b, P, alpha, theta, rho, leaf, R = case
    sys = H.hfsem_assemble([H.make_problem(h, P, alpha, theta, rho, a=a, b=b, matvec=1)])
    adm = H.ADM_MAX if rule == "max" else H.ADM_MIN
    fac = H.hfsem_hlu_factor(sys, H.hopts(R=R, lam=1.0, tol_hlu=0.0, precision=H.PREC_FP64,
                                          leaf_elems=leaf, kmax=48, admissibility=adm))
    m = Mesh(h, a, b)
    At, _ = hmatrix_dense(m, P, alpha, theta, system_full(m, P, alpha, theta, rho), R, 1.0, leaf,
                          rule=rule)
    rng = np.random.default_rng(11)
    Nd = n_dof(len(h), P)
    r = rng.standard_normal((3, Nd))
    y = H.hfsem_precond_apply(fac, np.ascontiguousarray(r.ravel()), nrhs=3).reshape(3, Nd)
    ref, _ = dense_solve(At, r.T)
    assert rel_err(y, ref.T) < 1e-9


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_hlu_mixed_is_a_good_preconditioner(lib, case):
    name, h, a, b, P, alpha, theta, rho, leaf, R = case
    sys = H.hfsem_assemble([H.make_problem(h, P, alpha, theta, rho, a=a, b=b, matvec=1)])
    fac = H.hfsem_hlu_factor(sys, H.hopts(R=R, tol_hlu=1e-3, precision=H.PREC_MIXED,
                                          leaf_elems=leaf))
    m = Mesh(h, a, b)
    Nd = n_dof(len(h), P)
    A = system_full(m, P, alpha, theta, rho)[:Nd, :Nd]
    rng = np.random.default_rng(5)
    x = rng.standard_normal(Nd)
    y = H.hfsem_precond_apply(fac, A @ x)
    # M^-1 A x should be close to x
    assert rel_err(y, x) < 0.2


@pytest.mark.parametrize("prec", [H.PREC_FP64, H.PREC_MIXED])
def test_preconditioned_solve_config1(lib, prec):
    p = W.config1()
    sys = H.hfsem_assemble([H.make_problem(p.h, p.P, p.alpha, p.theta, p.rho, c1=p.c1, c2=p.c2)])
    fac = H.hfsem_hlu_factor(sys, H.hopts(R=4, precision=prec))
    X, st, code = H.hfsem_solve(sys, fac, [H.rhs_frac_powers([p.rhs[0]])], tol=1e-15,
                                max_iter=100, allow_fail=True)
    Xo, _ = solve_problem(Mesh(p.h, 0, 1), p.P, p.alpha, p.theta, p.rho, p.c1, p.c2,
                          ("frac_powers", p.rhs[0]))
    assert rel_err(X, Xo) < 1e-10, (st, rel_err(X, Xo))
    assert st[0]["iters"] <= 20


def test_preconditioned_solve_batch_mixed_meshes(lib):
    # several instances of different shape in one batched call
    rng = np.random.default_rng(2)
    insts = [("uniform", W.mesh_uniform(40), 5, 1.4, 0.3, 1.0),
             ("graded3", W.mesh_graded(33, 3.0), 4, 1.7, 0.8, 0.0),
             ("geo2", W.mesh_geometric_two_sided(24, 0.5), 6, 1.2, 0.5, 2.0)]
    probs, rhs, refs = [], [], []
    for name, h, P, alpha, theta, rho in insts:
        probs.append(H.make_problem(h, P, alpha, theta, rho))
        coeffs = W.legendre_rhs(12, rng)
        rhs.append(H.rhs_legendre([coeffs]))
        Xo, _ = solve_problem(Mesh(h, 0, 1), P, alpha, theta, rho, 0.0, 0.0,
                              ("legendre_ab", coeffs))
        refs.append(Xo)
    sys = H.hfsem_assemble(probs)
    fac = H.hfsem_hlu_factor(sys, H.hopts(R=6, precision=H.PREC_MIXED))
    X, st, code = H.hfsem_solve(sys, fac, rhs, tol=1e-15, max_iter=100, allow_fail=True)
    for k, Xk in enumerate(H.split(sys, X)):
        assert rel_err(Xk[:, 0], refs[k]) < 1e-10, (k, st[k])


def test_factor_is_tied_to_its_system(lib):
    # a factor is valid only for the system it was built from, and one built
    # for inspection only cannot precondition
    h = W.mesh_uniform(12)
    s1 = H.hfsem_assemble([H.make_problem(h, 3, 1.5, 0.5, 1.0)])
    s2 = H.hfsem_assemble([H.make_problem(h, 3, 1.5, 0.5, 1.0)])
    f1 = H.hfsem_hlu_factor(s1, H.hopts(R=4))
    rhs = [H.rhs_legendre([np.array([1.0, 0.5])])]
    X, st, code = H.hfsem_solve(s2, f1, rhs, tol=1e-12, max_iter=20, allow_fail=True)
    assert code == H.HFSEM_ERR_INVALID_ARG
    fb = H.hfsem_hlu_factor(s1, H.hopts(R=4, build_only=1))
    X, st, code = H.hfsem_solve(s1, fb, rhs, tol=1e-12, max_iter=20, allow_fail=True)
    assert code == H.HFSEM_ERR_INVALID_ARG
    X, st, code = H.hfsem_solve(s1, f1, rhs, tol=1e-12, max_iter=20)
    assert code == H.HFSEM_OK


def test_direct_hmatrix_solve_falls_behind_with_n(lib):
    # Sec. 5, Example 1 (graded x_i = 10 (i/N)^5, alpha = 1.6, theta = 1,
    # rho = 0, P = 3, R = 3, Tol_HLU = 1e-13): the H-matrix approximation
    # system solved directly (hfsem_hlu_solve) matches the oracle's dense
    # solve of A~, and its error against the exact discrete solution grows
    # with N, while BiCGSTAB preconditioned by the same factor reaches the
    # exact discrete solution at every N
    a, b, gam, alpha, P, R = 0.0, 10.0, 0.8, 1.6, 3, 3
    terms, _, _ = W.manufactured_rhs([1.0, -(b - a) ** (1 - gam)], alpha, 1.0, 0.0, a, b,
                                     powers=[1.0, gam])
    errs = []
    for N in (50, 100, 200, 400):
        h = W.mesh_graded(N, 5.0, a, b)
        m = Mesh(h, a, b)
        Nd = n_dof(N, P)
        A = system_full(m, P, alpha, 1.0, 0.0)
        Xo, _ = solve_problem(m, P, alpha, 1.0, 0.0, 0.0, 0.0, ("frac_powers", terms), A_full=A)
        At, _ = hmatrix_dense(m, P, alpha, 1.0, A, R, 1.0, leaf=4)
        G = load_frac_powers(m, P, terms)[:Nd]
        XHo, _ = dense_solve(At, G)
        sys = H.hfsem_assemble([H.make_problem(h, P, alpha, 1.0, 0.0, a=a, b=b)])
        fac = H.hfsem_hlu_factor(sys, H.hopts(R=R, lam=1.0, tol_hlu=1e-13, precision=H.PREC_FP64,
                                              leaf_elems=4))
        XH = H.hfsem_hlu_solve(sys, fac, [H.rhs_frac_powers([terms])])
        assert rel_err(XH, XHo) < 1e-9, N
        XK, st, code = H.hfsem_solve(sys, fac, [H.rhs_frac_powers([terms])], tol=1e-14, max_iter=50)
        assert code == H.HFSEM_OK and rel_err(XK, Xo) < 1e-10, (N, st)
        errs.append(rel_err(XH, Xo))
    # measured with the oracle: 2.8e-4, 1.5e-2, 8.0e-2, 2.4e-1
    assert all(e1 < e2 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[-1] > 1e-2, errs


@pytest.mark.parametrize("prec", [H.PREC_MIXED, H.PREC_FP64])
def test_wide_cluster_factor_matches_the_batched_one(lib, prec):
    # one large instance alone runs its H-LU program on a cluster of 16 CTAs,
    # the same instance in a batch of three on clusters of 8: the ops of a
    # wave are independent and each op's arithmetic does not depend on the
    # CTA that runs it, so the preconditioned solves agree to rounding
    h = W.mesh_graded(1024, 2.0)
    P = 9                                  # N_d = 9215
    prob = H.make_problem(h, P, 1.4, 0.6, 0.5, matvec=H.MATVEC_HMATRIX)
    opts = H.hopts(R=8, lam=1.0, tol_hlu=1e-3, precision=prec, admissibility=H.ADM_MIN)
    terms = [[(1.0, 0.5, "a"), (-0.5, 1.5, "b")]]
    alone = H.hfsem_assemble([prob])
    fa = H.hfsem_hlu_factor(alone, opts)
    Xa, sa, ca = H.hfsem_solve(alone, fa, [H.rhs_frac_powers(terms)], tol=1e-14, max_iter=60)
    batch = H.hfsem_assemble([prob, prob, prob])
    fb = H.hfsem_hlu_factor(batch, opts)
    Xb, sb, cb = H.hfsem_solve(batch, fb, [H.rhs_frac_powers(terms)] * 3, tol=1e-14, max_iter=60)
    assert ca == H.HFSEM_OK and cb == H.HFSEM_OK
    assert sa[0]["iters"] == sb[0]["iters"], (sa, sb)
    xb = H.split(batch, Xb)
    for k in range(3):
        assert rel_err(xb[k][:, 0], Xa) < 1e-13, k


@pytest.mark.parametrize("prec", [H.PREC_MIXED, H.PREC_FP64])
def test_rhs_chunks_split_over_clusters(lib, prec):
    # one instance with 16 right-hand sides: its H-solves split the chunks of
    # right-hand sides over several clusters; in a batch of 16 copies every
    # instance's chunks run on its own cluster in turn.  Same arithmetic per
    # chunk, so the solutions agree to rounding
    h = W.mesh_graded(400, 2.0)
    prob = H.make_problem(h, 8, 1.7, 0.3, 1.0, matvec=H.MATVEC_HMATRIX)
    opts = H.hopts(R=8, lam=1.0, tol_hlu=1e-3, precision=prec, admissibility=H.ADM_MIN)
    terms = [[(1.0, 0.3 + 0.2 * k, "a"), (0.5 - 0.05 * k, 1.0 + 0.1 * k, "b")] for k in range(16)]
    rhs = H.rhs_frac_powers(terms)
    alone = H.hfsem_assemble([prob])
    fa = H.hfsem_hlu_factor(alone, opts)
    Xa, sa, ca = H.hfsem_solve(alone, fa, [rhs], tol=1e-14, max_iter=60)
    batch = H.hfsem_assemble([prob] * 16)
    fb = H.hfsem_hlu_factor(batch, opts)
    Xb, sb, cb = H.hfsem_solve(batch, fb, [rhs] * 16, tol=1e-14, max_iter=60)
    assert ca == H.HFSEM_OK and cb == H.HFSEM_OK
    xa = H.split(alone, Xa, 16)[0]
    for k, xb in enumerate(H.split(batch, Xb, 16)):
        for r in range(16):
            assert rel_err(xb[:, r], xa[:, r]) < 1e-14, (k, r)
    assert [s["iters"] for s in sa] == [s["iters"] for s in sb[:16]]


@pytest.mark.parametrize("prec", [H.PREC_MIXED, H.PREC_FP64])
def test_narrow_cluster_factor_matches_the_single_one(lib, prec):
    # a batch of 40 instances runs its H-LU programs on clusters of 4 CTAs,
    # one instance alone on a cluster of 8: same factor, same solutions
    h = W.mesh_geometric_two_sided(96, 0.6)
    prob = H.make_problem(h, 6, 1.25, 0.8, 0.2, matvec=H.MATVEC_HMATRIX)
    opts = H.hopts(R=8, lam=1.0, tol_hlu=1e-3, precision=prec, admissibility=H.ADM_MIN)
    rhs = H.rhs_frac_powers([[(1.0, 0.7, "a"), (2.0, 0.2, "b")]])
    alone = H.hfsem_assemble([prob])
    fa = H.hfsem_hlu_factor(alone, opts)
    Xa, sa, ca = H.hfsem_solve(alone, fa, [rhs], tol=1e-14, max_iter=60)
    batch = H.hfsem_assemble([prob] * 40)
    fb = H.hfsem_hlu_factor(batch, opts)
    Xb, sb, cb = H.hfsem_solve(batch, fb, [rhs] * 40, tol=1e-14, max_iter=60)
    assert ca == H.HFSEM_OK and cb == H.HFSEM_OK
    for k, xb in enumerate(H.split(batch, Xb)):
        assert rel_err(xb[:, 0], Xa) < 1e-14, k
    assert all(s["iters"] == sa[0]["iters"] for s in sb)
