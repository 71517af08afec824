"""GPU parity of the assembled operator and load vector against the oracle
(element by element), through the C ABI."""
import numpy as np
import pytest

from oracle.assemble import system_full
from oracle.basis import Mesh, n_dof
from oracle.load import load_frac_powers, load_legendre_ab
from oracle.solve import solve_problem
from paper_1808_02937_gb300 import hfsem as H
from paper_1808_02937_gb300 import workloads as W
from tests._common import ensure_built, rel_err

pytestmark = pytest.mark.gpu


def _cases():
    g5 = W.mesh_graded(12, 5.0, 0.0, 10.0)
    return [
        # (name, h, a, b, P, alpha, theta, rho, matvec)
        ("uniform-auto", W.mesh_uniform(16), 0.0, 1.0, 4, 1.5, 0.5, 0.0, 0),
        ("uniform-dense", W.mesh_uniform(16), 0.0, 1.0, 4, 1.5, 0.5, 0.0, 1),
        ("uniform-P1", W.mesh_uniform(9), 0.0, 1.0, 1, 1.3, 0.2, 1.0, 0),
        ("uniform-P8-rho", W.mesh_uniform(7, -1.0, 1.0), -1.0, 1.0, 8, 1.8, 0.3, 2.0, 0),
        ("geo1-toep", W.mesh_geometric_one_sided(10, 0.8), 0.0, 1.0, 3, 1.4, 0.7, 0.5, 2),
        ("geo1-dense", W.mesh_geometric_one_sided(10, 0.8), 0.0, 1.0, 3, 1.4, 0.7, 0.5, 1),
        ("geo2", W.mesh_geometric_two_sided(12, 0.5), 0.0, 1.0, 5, 1.3, 0.7, 1.0, 0),
        ("graded5", g5, 0.0, 10.0, 3, 1.6, 1.0, 0.0, 0),
        ("graded2-theta0", W.mesh_graded(9, 2.0), 0.0, 1.0, 6, 1.1, 0.0, 0.3, 0),
        ("one-element", np.array([2.0]), 0.0, 2.0, 5, 1.7, 0.4, 1.0, 0),
        ("two-elements-P16", W.mesh_uniform(2), 0.0, 1.0, 16, 1.25, 0.6, 0.0, 0),
        ("ragged-P7", W.mesh_graded(23, 3.0), 0.0, 1.0, 7, 1.45, 0.35, 0.8, 0),
        # register tiles of the dense operator for P up to 24 and 32
        ("graded-P20", W.mesh_graded(5, 2.0), 0.0, 1.0, 20, 1.35, 0.55, 0.2, 1),
        ("dense-P32", W.mesh_uniform(3), 0.0, 1.0, 32, 1.65, 0.8, 0.0, 1),
    ]


def test_mixed_degree_batch_dense_operator(lib):
    # one batch, dense instances of P = 3 and P = 14 (the larger register tile
    # serves both), against each instance's oracle operator
    rng = np.random.default_rng(11)
    cases = [(W.mesh_graded(17, 2.0), 3, 1.2, 0.1, 0.5), (W.mesh_graded(6, 3.0), 14, 1.7, 0.9, 0.0),
             (W.mesh_geometric_two_sided(10, 0.6), 5, 1.5, 0.5, 1.0)]
    sys = H.hfsem_assemble([H.make_problem(h, P, al, th, rho, matvec=1)
                            for h, P, al, th, rho in cases])
    xs = [rng.standard_normal((3, n_dof(len(h), P))) for h, P, *_ in cases]
    y = H.hfsem_apply(sys, np.concatenate([x.ravel() for x in xs]), nrhs=3)
    off = 0
    for (h, P, al, th, rho), x in zip(cases, xs):
        Nd = n_dof(len(h), P)
        A = system_full(Mesh(h, 0.0, 1.0), P, al, th, rho)[:Nd, :Nd]
        got = y[off: off + 3 * Nd].reshape(3, Nd)
        off += 3 * Nd
        for r in range(3):
            ref = A @ x[r]
            # rounding of a sum of products: O(eps sum_j |A_ij x_j|) per row
            bound = 1e-13 * (np.abs(A) @ np.abs(x[r]))
            assert np.all(np.abs(got[r] - ref) <= bound), np.max(np.abs(got[r] - ref) / bound)


@pytest.fixture(scope="module")
def lib():
    return ensure_built()


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_operator_entries_match_oracle(lib, case):
    name, h, a, b, P, alpha, theta, rho, mv = case
    prob = H.make_problem(h, P, alpha, theta, rho, a=a, b=b, matvec=mv)
    sys = H.hfsem_assemble([prob])
    Nd = n_dof(len(h), P)
    A_ref = system_full(Mesh(h, a, b), P, alpha, theta, rho)[:Nd, :Nd]
    # columns of A by applying to unit vectors, up to 64 at a time
    A_gpu = np.zeros((Nd, Nd))
    for c0 in range(0, Nd, 64):
        k = min(64, Nd - c0)
        E = np.zeros((k, Nd))
        E[np.arange(k), c0 + np.arange(k)] = 1.0
        Y = H.hfsem_apply(sys, np.ascontiguousarray(E.ravel()), nrhs=k)
        A_gpu[:, c0:c0 + k] = Y.reshape(k, Nd).T
    scale = np.abs(A_ref).max()
    err = np.abs(A_gpu - A_ref).max() / scale
    assert err < 5e-13, (name, err)


def test_toeplitz_equals_dense_at_size(lib):
    # N = 1024 uniform, P = 8: the FFT operator against the dense one
    rng = np.random.default_rng(7)
    h = W.mesh_uniform(1024)
    probs = [H.make_problem(h, 8, al, th, 1.0, matvec=mv)
             for al, th in ((1.2, 0.0), (1.8, 0.5)) for mv in (2, 1)]
    sys = H.hfsem_assemble(probs)
    Nd = 1024 * 8 - 1
    x1 = rng.standard_normal(Nd)
    x = np.concatenate([x1] * 4)
    y = H.hfsem_apply(sys, x).reshape(4, Nd)
    for k in (0, 2):
        # the dense operator's rounding is O(eps * sum |A_ij x_j|)
        assert rel_err(y[k], y[k + 1]) < 1e-11


@pytest.mark.parametrize("side_terms", [
    [(1.0, -0.5, "a"), (2.0, 0.3, "b")],
    [(-1.3, 1 - 1.6, "a"), (0.7, 2 - 1.6, "a"), (0.25, 3.0, "b"), (1.0, 0.0, "a")],
])
@pytest.mark.parametrize("mesh", ["uniform", "graded5", "geo2"])
def test_load_vector_frac_powers(lib, side_terms, mesh):
    h = {"uniform": W.mesh_uniform(10), "graded5": W.mesh_graded(14, 5.0),
         "geo2": W.mesh_geometric_two_sided(16, 0.4)}[mesh]
    P = 6
    prob = H.make_problem(h, P, 1.5, 0.5, 0.0)
    sys = H.hfsem_assemble([prob])
    G = H.hfsem_load_vector(sys, [H.rhs_frac_powers([side_terms])])
    ref = load_frac_powers(Mesh(h, 0.0, 1.0), P, side_terms)[: n_dof(len(h), P)]
    assert np.abs(G - ref).max() < 1e-12 * np.abs(ref).max()


def test_load_vector_legendre(lib):
    rng = np.random.default_rng(3)
    coeffs = W.legendre_rhs(32, rng)
    h = W.mesh_graded(20, 2.0, -1.0, 2.0)
    prob = H.make_problem(h, 9, 1.5, 0.5, 0.0, a=-1.0, b=2.0)
    sys = H.hfsem_assemble([prob])
    G = H.hfsem_load_vector(sys, [H.rhs_legendre([coeffs])])
    ref = load_legendre_ab(Mesh(h, -1.0, 2.0), 9, coeffs)[: n_dof(20, 9)]
    assert np.abs(G - ref).max() < 1e-13 * np.abs(ref).max()


def test_lifted_load_vector(lib):
    h = W.mesh_graded(8, 2.0)
    P, alpha, theta, rho, c1, c2 = 4, 1.4, 0.3, 0.7, 1.0, 2.0
    terms = [(1.0, 0.0, "a"), (0.5, 1 - alpha, "b")]
    prob = H.make_problem(h, P, alpha, theta, rho, c1=c1, c2=c2)
    sys = H.hfsem_assemble([prob])
    G = H.hfsem_load_vector(sys, [H.rhs_frac_powers([terms])], lifted=1)
    m = Mesh(h, 0.0, 1.0)
    Nd = n_dof(8, P)
    A = system_full(m, P, alpha, theta, rho)
    ref = load_frac_powers(m, P, terms)[:Nd] - A[:Nd, Nd:] @ np.array([c1, c2])
    assert np.abs(G - ref).max() < 1e-12 * np.abs(ref).max()


def test_unpreconditioned_solve_config1(lib):
    p = W.config1()
    prob = H.make_problem(p.h, p.P, p.alpha, p.theta, p.rho, c1=p.c1, c2=p.c2)
    sys = H.hfsem_assemble([prob])
    X, st, code = H.hfsem_solve(sys, None, [H.rhs_frac_powers([p.rhs[0]])], tol=1e-15,
                                max_iter=400, allow_fail=True)
    Xo, _ = solve_problem(Mesh(p.h, 0, 1), p.P, p.alpha, p.theta, p.rho, p.c1, p.c2,
                          ("frac_powers", p.rhs[0]))
    assert rel_err(X, Xo) < 1e-10, (st, rel_err(X, Xo))
