"""The FP64 H-matrix operator (HFSEM_MATVEC_HMATRIX: exact near-field pairs,
Taylor rank 24 with the min-diameter rule at lambda = 1, Sec. 3 at a rank
where the Lemma's bound (1/3)^24 is below FP64 rounding) against the oracle:

* its entries (applied to unit vectors) against the oracle's dense A;
* its product on random vectors against A x, in a batch that mixes it with
  dense and Toeplitz instances;
* the lifted load vector (boundary values) against the oracle's;
* solves preconditioned by an H-LU of the same near field reach the oracle's
  exact discrete solution;
* a preconditioner whose near field is not stored is refused (UNSUPPORTED);
* the largest graded request (N = 4096, P = 16, 16 rhs) reproduces the
  manufactured polynomials.
"""
import numpy as np
import pytest

from oracle.assemble import system_full
from oracle.basis import Mesh, n_dof
from oracle.load import load_frac_powers
from paper_1808_02937_gb300 import hfsem as H
from paper_1808_02937_gb300 import workloads as W
from tests._common import ensure_built, rel_err
from tests._oracle_pool import oracle_solve_many
from tests.test_oracle_solve import expected_coeffs

pytestmark = pytest.mark.gpu

HM = H.MATVEC_HMATRIX


@pytest.fixture(scope="module")
def lib():
    return ensure_built()


CASES = [
    # name, h, P, alpha, theta, rho
    ("graded2", W.mesh_graded(60, 2.0), 4, 1.3, 0.6, 0.5),
    ("graded3-P8", W.mesh_graded(40, 3.0), 8, 1.75, 0.2, 0.0),
    ("geo2", W.mesh_geometric_two_sided(48, 0.45), 5, 1.5, 1.0, 1.0),
    ("graded-P2", W.mesh_graded(150, 2.0), 2, 1.1, 0.0, 1.5),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
def test_hmatrix_operator_entries_match_oracle(lib, case):
    name, h, P, alpha, theta, rho = case
    sys_ = H.hfsem_assemble([H.make_problem(h, P, alpha, theta, rho, matvec=HM)])
    Nd = n_dof(len(h), P)
    A = system_full(Mesh(h, 0.0, 1.0), P, alpha, theta, rho)[:Nd, :Nd]
    G = np.zeros((Nd, Nd))
    for c0 in range(0, Nd, 64):
        k = min(64, Nd - c0)
        E = np.zeros((k, Nd))
        E[np.arange(k), c0 + np.arange(k)] = 1.0
        G[:, c0:c0 + k] = H.hfsem_apply(sys_, np.ascontiguousarray(E.ravel()), nrhs=k).reshape(k, Nd).T
    err = np.abs(G - A).max() / np.abs(A).max()
    assert err < 5e-13, (name, err)


def test_hmatrix_operator_in_mixed_batch(lib):
    rng = np.random.default_rng(5)
    specs = [(W.mesh_graded(300, 2.0), 6, 1.4, 0.3, 1.0, HM),
             (W.mesh_uniform(64), 4, 1.6, 0.5, 0.0, H.MATVEC_AUTO),
             (W.mesh_geometric_two_sided(120, 0.5), 3, 1.9, 0.8, 0.2, HM),
             (W.mesh_graded(30, 3.0), 5, 1.2, 0.1, 0.7, H.MATVEC_DENSE)]
    sys_ = H.hfsem_assemble([H.make_problem(h, P, a, t, r, matvec=mv) for h, P, a, t, r, mv in specs])
    xs = [rng.standard_normal((2, n_dof(len(h), P))) for h, P, *_ in specs]
    y = H.hfsem_apply(sys_, np.concatenate([x.ravel() for x in xs]), nrhs=2)
    off = 0
    for (h, P, a, t, r, mv), x in zip(specs, xs):
        Nd = n_dof(len(h), P)
        A = system_full(Mesh(h, 0.0, 1.0), P, a, t, r)[:Nd, :Nd]
        got = y[off: off + 2 * Nd].reshape(2, Nd)
        off += 2 * Nd
        for k in range(2):
            ref = A @ x[k]
            bound = 1e-12 * (np.abs(A) @ np.abs(x[k]))
            assert np.all(np.abs(got[k] - ref) <= bound), (mv, np.max(np.abs(got[k] - ref) / bound))


def test_hmatrix_lifted_load_vector(lib):
    h = W.mesh_graded(70, 2.0)
    P, alpha, theta, rho, c1, c2 = 5, 1.45, 0.35, 0.8, 1.5, -0.75
    terms = [(1.0, 0.0, "a"), (0.5, 1 - alpha, "b")]
    sys_ = H.hfsem_assemble([H.make_problem(h, P, alpha, theta, rho, c1=c1, c2=c2, matvec=HM)])
    G = H.hfsem_load_vector(sys_, [H.rhs_frac_powers([terms])], lifted=1)
    m = Mesh(h, 0.0, 1.0)
    Nd = n_dof(len(h), P)
    A = system_full(m, P, alpha, theta, rho)
    ref = load_frac_powers(m, P, terms)[:Nd] - A[:Nd, Nd:] @ np.array([c1, c2])
    assert np.abs(G - ref).max() < 1e-12 * np.abs(ref).max()


OPTS = dict(R=8, lam=1.0, tol_hlu=1e-3, admissibility=H.ADM_MIN)


@pytest.mark.parametrize("prec", [H.PREC_MIXED, H.PREC_FP64])
def test_hmatrix_solves_reach_oracle(lib, prec):
    p3 = W.config3()        # two-sided geometric q = 0.5, N = 256, P = 16
    g = W.mesh_graded(300, 2.0)
    rng = np.random.default_rng(8)
    coef = W.legendre_rhs(32, rng)
    probs = [H.make_problem(p3.h, p3.P, p3.alpha, p3.theta, p3.rho, matvec=HM),
             H.make_problem(g, 7, 1.35, 0.65, 1.0, c1=0.5, c2=-1.0, matvec=HM)]
    sys_ = H.hfsem_assemble(probs)
    fac = H.hfsem_hlu_factor(sys_, H.hopts(precision=prec, **OPTS))
    X, st, code = H.hfsem_solve(sys_, fac, [H.rhs_legendre([p3.rhs[0]]), H.rhs_legendre([coef])],
                                tol=1e-14, max_iter=80)
    assert code == H.HFSEM_OK, st
    ref = oracle_solve_many([(p3.h, 0.0, 1.0, p3.P, p3.alpha, p3.theta, p3.rho, 0.0, 0.0,
                              ("legendre_ab", p3.rhs[0])),
                             (g, 0.0, 1.0, 7, 1.35, 0.65, 1.0, 0.5, -1.0, ("legendre_ab", coef))])
    parts = H.split(sys_, X)
    for k in range(2):
        assert rel_err(parts[k][:, 0], ref[k]) < 1e-10, (k, st)


def test_preconditioner_outside_stored_near_field_refused(lib):
    # the paper's max-diameter rule needs far more near-field pairs on a
    # geometric mesh than the operator stores
    sys_ = H.hfsem_assemble([H.make_problem(W.mesh_geometric_two_sided(256, 0.7), 4, 1.5, 0.5, 1.0,
                                            matvec=HM)])
    with pytest.raises(H.HfsemError) as e:
        H.hfsem_hlu_factor(sys_, H.hopts(R=8, admissibility=H.ADM_MAX))
    assert e.value.code == H.HFSEM_ERR_UNSUPPORTED


def test_largest_graded_request_with_hmatrix_operator(lib):
    p = W.config5_max_request("graded")
    assert p.Nd == 65535 and len(p.rhs) == 16
    sys_ = H.hfsem_assemble([H.make_problem(p.h, p.P, p.alpha, p.theta, p.rho, matvec=HM)])
    fac = H.hfsem_hlu_factor(sys_, H.hopts(precision=H.PREC_MIXED, **OPTS))
    X, st, code = H.hfsem_solve(sys_, fac, [H.rhs_frac_powers(p.rhs)], tol=1e-14, max_iter=100)
    assert code == H.HFSEM_OK, st
    parts = H.split(sys_, X, nrhs=16)[0]
    for r, u in enumerate(p.u_exact):
        Xe = expected_coeffs(Mesh(p.h, 0.0, 1.0), p.P, np.polynomial.Polynomial(u))
        assert rel_err(parts[:, r], Xe) < 1e-10, r
