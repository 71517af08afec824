"""Pins for the oracle's whole discrete solve and for the manufactured
right-hand sides: exact reproduction of solutions that lie in the SEM space,
the weak form checked by QUADPACK, and h/p convergence (Sec. 5)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle.basis import Mesh, legendre_all, local_values, n_dof
from oracle.quadrature import gauss_legendre
from oracle.solve import solve_problem
from paper_1808_02937_gb300 import workloads as W


def expected_coeffs(mesh, P, u):
    """Coefficients of a polynomial u (numpy Polynomial in x - a) in the SEM
    basis: hats take nodal values, bubbles the Legendre coefficients of u'
    (psi_p' = -(2p+1) L_p)."""
    N = mesh.N
    du = u.deriv()
    xq, wq = gauss_legendre(30)
    L = legendre_all(P, xq)
    bub = np.zeros((N, P - 1))
    for e in range(N):
        y = mesh.dl[e] + 0.5 * mesh.h[e] * (1 + xq)
        for p in range(1, P):
            bub[e, p - 1] = -(mesh.h[e] / 4) * np.sum(wq * du(y) * L[p])
    return np.concatenate([bub.ravel(), u(mesh.dl[1:N])])


def evaluate(mesh, P, X, c1, c2, y):
    """u_N^P at offsets y = x - a."""
    N = mesh.N
    hats = np.concatenate([[c1], X[N * (P - 1):], [c2]])
    bub = X[: N * (P - 1)].reshape(N, P - 1)
    e = np.clip(np.searchsorted(mesh.dl, y, side="right") - 1, 0, N - 1)
    xi = -1 + 2 * (y - mesh.dl[e]) / mesh.h[e]
    out = np.empty_like(y)
    for k in range(len(y)):
        V = local_values(P, np.array([xi[k]]))[:, 0]
        out[k] = hats[e[k]] * V[0] + hats[e[k] + 1] * V[1] + bub[e[k]] @ V[2:]
    return out


def test_config1_exact_reproduction():
    p = W.config1()
    mesh = Mesh(p.h, p.a, p.b)
    X, info = solve_problem(mesh, p.P, p.alpha, p.theta, p.rho, p.c1, p.c2,
                            ("frac_powers", p.rhs[0]))
    Xe = expected_coeffs(mesh, p.P, np.polynomial.Polynomial(p.u_exact))
    assert np.linalg.norm(X - Xe) / np.linalg.norm(Xe) < 1e-12
    assert info["corr"] < 1e-14


def test_nonzero_boundary_values_reproduced():
    # u = 1 + 2x - x^3 on a graded mesh: u(0) = 1, u(1) = 2 enter by lifting
    alpha, theta, rho, P = 1.4, 0.3, 0.7, 3
    u = [1.0, 2.0, 0.0, -1.0]
    terms, c1, c2 = W.manufactured_rhs(u, alpha, theta, rho, 0.0, 1.0)
    assert (c1, c2) == (1.0, 2.0)
    mesh = Mesh(W.mesh_graded(5, 2.0))
    X, _ = solve_problem(mesh, P, alpha, theta, rho, c1, c2, ("frac_powers", terms))
    Xe = expected_coeffs(mesh, P, np.polynomial.Polynomial(u))
    assert np.linalg.norm(X - Xe) / np.linalg.norm(Xe) < 1e-12


def test_constant_solution():
    # u = c: u' = 0, so f = rho c and every hat coefficient is c
    mesh = Mesh(W.mesh_geometric_one_sided(6, 0.6))
    c, rho = 1.7, 2.5
    X, _ = solve_problem(mesh, 4, 1.7, 0.4, rho, c, c, ("frac_powers", [(rho * c, 0.0, "a")]))
    N, P = 6, 4
    assert np.allclose(X[N * (P - 1):], c, atol=1e-13)
    assert np.allclose(X[: N * (P - 1)], 0.0, atol=1e-13)


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
@pytest.mark.parametrize("u,theta,rho", [([0, 0, 1, -2, 1], 0.3, 0.7),
                                         ([1, 2, 0, -1], 0.8, 0.0)])
def test_manufactured_rhs_weak_form(u, theta, rho):
    # (f, v) = theta (aI u', v') + (1-theta) (xI u', v') + rho (u, v) for v in H^1_0
    alpha, a, b = 1.4, 0.0, 1.0
    terms, _, _ = W.manufactured_rhs(u, alpha, theta, rho, a, b)
    U = np.polynomial.Polynomial(u)
    dU = U.deriv()
    g0 = 1 / math.gamma(2 - alpha)
    for v in (np.polynomial.Polynomial([0, 1, -1]), np.polynomial.Polynomial([0, 0, 1, -1])):
        dv = v.deriv()
        left = lambda t: integrate.quad(dU, a, t, weight="alg", wvar=(0, 1 - alpha))[0] if t > a else 0.0
        right = lambda t: integrate.quad(dU, t, b, weight="alg", wvar=(1 - alpha, 0))[0] if t < b else 0.0
        B = g0 * integrate.quad(lambda t: dv(t) * (theta * left(t) + (1 - theta) * right(t)),
                                a, b, epsabs=1e-13, limit=100)[0]
        B += rho * integrate.quad(lambda t: U(t) * v(t), a, b)[0]
        F = 0.0
        for coef, mu, side in terms:
            wv = (mu, 0.0) if side == "a" else (0.0, mu)
            F += coef * integrate.quad(v, a, b, weight="alg", wvar=wv)[0]
        assert abs(F - B) < 1e-9 * max(1.0, abs(B))


def _example1(N, P):
    # Example 1: u = (x-a) - (b-a)^(1-gamma) (x-a)^gamma, theta = 1, rho = 0,
    # a = 0, b = 10, gamma = 0.8, graded mesh x_i = (i/N)^5 (b-a); alpha = 1.6
    a, b, gam, alpha = 0.0, 10.0, 0.8, 1.6
    coeffs = [1.0, -(b - a) ** (1 - gam)]
    terms, c1, c2 = W.manufactured_rhs(coeffs, alpha, 1.0, 0.0, a, b, powers=[1.0, gam])
    mesh = Mesh(W.mesh_graded(N, 5.0, a, b), a, b)
    X, _ = solve_problem(mesh, P, alpha, 1.0, 0.0, 0.0, 0.0, ("frac_powers", terms))
    y = np.linspace(0, 10, 401)[1:-1]
    uex = y - (b - a) ** (1 - gam) * y ** gam
    return np.abs(evaluate(mesh, P, X, 0.0, 0.0, y) - uex).max()


def test_example1_h_refinement():
    errs = [_example1(N, 3) for N in (8, 16, 32)]
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-3


def test_example1_p_refinement():
    errs = [_example1(16, P) for P in (2, 3, 4, 5)]
    assert all(e1 > e2 for e1, e2 in zip(errs, errs[1:]))
