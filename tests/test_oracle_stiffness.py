"""Pins for the oracle's dense stiffness / mass assembly (Sec. 2.2).

Each pin comes from outside the oracle: QUADPACK brute force, a closed form
for the fractional integral of a Legendre polynomial, the alpha -> 1 and
alpha -> 2 limits of the kernel, the reflection symmetry S_r = S_l^T, the
theta = 1/2 symmetry and coercivity (Thm 1), and mass-matrix closed forms."""
import math
import warnings

import numpy as np
import pytest
from scipy import integrate, special

from oracle.assemble import (mass, pair_self, pair_separated, pair_touch,
                             stiffness_left, stiffness_right, system_full)
from oracle.basis import Mesh, global_index, local_derivs, local_values, n_dof


def _phi_d(P, k, x0, h):
    """Physical derivative of local function k of the element [x0, x0+h]."""
    return lambda t: (2.0 / h) * local_derivs(P, np.array([(2 * (t - x0) / h) - 1.0]))[k, 0]


def _brute_pair(mesh, P, alpha, e, f, a, b):
    x = mesh.dl
    g0 = 1.0 / math.gamma(2 - alpha)
    dpa = _phi_d(P, a, x[e], mesh.h[e])
    dpb = _phi_d(P, b, x[f], mesh.h[f])

    def inner(t):
        hi = min(t, x[f + 1])
        if e == f:
            v, _ = integrate.quad(dpb, x[f], hi, weight="alg", wvar=(0.0, 1.0 - alpha),
                                  epsabs=1e-14, epsrel=1e-12, limit=100)
            return v
        v, _ = integrate.quad(lambda s: (t - s) ** (1 - alpha) * dpb(s), x[f], hi,
                              epsabs=1e-14, epsrel=1e-12, limit=100)
        return v
    v, _ = integrate.quad(lambda t: dpa(t) * inner(t), x[e], x[e + 1],
                          epsabs=1e-13, epsrel=1e-11, limit=100)
    return g0 * v


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
@pytest.mark.parametrize("e,f", [(1, 1), (2, 1), (3, 1)])
def test_pairs_against_quadpack(e, f):
    P, alpha = 3, 1.35
    mesh = Mesh(np.array([0.3, 0.7, 0.45, 1.1]))
    if e == f:
        K = pair_self(mesh.h[e], P, alpha)
    elif e == f + 1:
        K = pair_touch(mesh.h[e], mesh.h[f], P, alpha)
    else:
        K = pair_separated(mesh.h[e], mesh.h[f], mesh.gap(f, e), P, alpha)
    scale = np.abs(K).max()
    # every entry for the cheap pairs, a spread sample for the touching pair
    entries = ([(a, b) for a in range(P + 1) for b in range(P + 1)] if e != f + 1
               else [(0, 0), (1, 1), (1, 2), (2, 3), (3, 0)])
    for a, b in entries:
        ref = _brute_pair(mesh, P, alpha, e, f, a, b)
        assert abs(K[a, b] - ref) < 2e-10 * scale, (a, b, K[a, b], ref)


@pytest.mark.parametrize("alpha", [1.1, 1.5, 1.85])
def test_self_pair_against_jacobi_identity(alpha):
    # int_{-1}^{xi} (xi-eta)^(1-alpha) L_n(eta) deta
    #   = Gamma(2-alpha) n!/Gamma(n+3-alpha) (1+xi)^(2-alpha) P_n^(alpha-2, 2-alpha)(xi)
    P = 7
    xq, wq = special.roots_jacobi(40, 0.0, 2.0 - alpha)      # weight (1+x)^(2-alpha)
    DL = np.zeros((P, P))
    for n in range(P):
        inner = (math.gamma(2 - alpha) * math.factorial(n) / math.gamma(n + 3 - alpha)
                 * special.eval_jacobi(n, alpha - 2.0, 2.0 - alpha, xq))
        for m in range(P):
            DL[m, n] = np.sum(wq * special.eval_legendre(m, xq) * inner)
    # local derivative basis in Legendre coefficients
    beta = np.zeros((P + 1, P))
    beta[0, 0], beta[1, 0] = -0.5, 0.5
    for p in range(1, P):
        beta[1 + p, p] = -(2 * p + 1)
    ref = beta @ DL @ beta.T / math.gamma(2 - alpha)          # gamma0 * ...
    K = pair_self(2.0, P, alpha)                               # h/2 = 1
    assert np.allclose(K, ref, rtol=0, atol=1e-13 * np.abs(ref).max())


def _interior(M, N, P):
    Nd = n_dof(N, P)
    return M[:Nd, :Nd]


def test_alpha_one_limit():
    # alpha = 1: gamma0 = 1, kernel 1, so S_l[i, j] = int phi_i' phi_j
    P = 4
    mesh = Mesh(np.array([0.2, 0.5, 0.3, 0.6, 0.4]))
    S = stiffness_left(mesh, P, 1.0)
    idx = global_index(mesh.N, P)
    ref = np.zeros_like(S)
    xq, wq = special.roots_legendre(12)
    for e in range(mesh.N):
        loc = (local_derivs(P, xq) * wq) @ local_values(P, xq).T
        ref[np.ix_(idx[e], idx[e])] += loc
    assert np.allclose(_interior(S, mesh.N, P), _interior(ref, mesh.N, P), atol=1e-13)


def test_alpha_two_limit():
    # alpha -> 2: gamma0 (t-s)^(1-alpha) -> delta, S_l -> int phi_i' phi_j'
    P = 3
    mesh = Mesh(np.array([0.25, 0.5, 0.25]))
    eps = 1e-6
    S = stiffness_left(mesh, P, 2.0 - eps)
    idx = global_index(mesh.N, P)
    ref = np.zeros_like(S)
    xq, wq = special.roots_legendre(8)
    for e in range(mesh.N):
        D = local_derivs(P, xq)
        ref[np.ix_(idx[e], idx[e])] += (2.0 / mesh.h[e]) * (D * wq) @ D.T
    Si, Ri = _interior(S, mesh.N, P), _interior(ref, mesh.N, P)
    assert np.abs(Si - Ri).max() < 1e-4 * np.abs(Ri).max()


@pytest.fixture(scope="module")
def graded():
    mesh = Mesh(np.diff((np.arange(8) / 7.0) ** 2.5) * 3.0, 0.0)
    P, alpha = 3, 1.45
    return mesh, P, alpha, stiffness_left(mesh, P, alpha), stiffness_right(mesh, P, alpha)


def test_right_is_transpose_of_left(graded):
    mesh, P, alpha, Sl, Sr = graded
    assert np.abs(Sr - Sl.T).max() < 1e-13 * np.abs(Sl).max()


def test_theta_half_symmetric_and_coercive(graded):
    mesh, P, alpha, Sl, Sr = graded
    Nd = n_dof(mesh.N, P)
    S = 0.5 * (Sl + Sr)[:Nd, :Nd]
    assert np.abs(S - S.T).max() < 1e-13 * np.abs(S).max()
    assert np.linalg.eigvalsh(S).min() > 0.0      # Thm 1


def test_quadratic_form_independent_of_theta(graded):
    mesh, P, alpha, Sl, Sr = graded
    Nd = n_dof(mesh.N, P)
    rng = np.random.default_rng(0)
    x = rng.standard_normal(Nd)
    vals = [x @ ((t * Sl + (1 - t) * Sr)[:Nd, :Nd]) @ x for t in (0.0, 0.3, 1.0)]
    assert vals[0] > 0
    assert np.allclose(vals, vals[0], rtol=1e-12)


def test_block_lower_structure(graded):
    # S_l[i, j] = 0 when every point of supp phi_i lies left of supp phi_j
    mesh, P, alpha, Sl, Sr = graded
    idx = global_index(mesh.N, P)
    for e in range(mesh.N):
        for f in range(e + 1, mesh.N):
            for a in range(P + 1):
                for b in range(P + 1):
                    gi, gj = idx[e, a], idx[f, b]
                    # skip the hat shared by e and f = e+1 (its support spans both)
                    if f == e + 1 and (a == 1 or b == 0):
                        continue
                    if gi == gj:
                        continue
                    # test function living only on e and left of trial support
                    if a >= 2 and b >= 2:
                        assert Sl[gi, gj] == 0.0


def test_mass_closed_form():
    P = 5
    mesh = Mesh(np.array([0.4, 0.9]))
    M = mass(mesh, P)
    idx = global_index(mesh.N, P)
    h = mesh.h[1]
    loc = M[np.ix_(idx[1], idx[1])]
    # element 1 shares its left hat with element 0: check the entries that
    # are local to element 1
    assert abs(loc[1, 1] - h / 3) < 1e-15                     # right hat (boundary node)
    for p in range(1, P):
        assert abs(loc[1 + p, 1 + p] - 0.5 * h * (2 / (2 * p - 1) + 2 / (2 * p + 3))) < 1e-15
        if p + 2 < P:
            assert abs(loc[1 + p, 3 + p] + 0.5 * h * 2 / (2 * p + 3)) < 1e-15
    assert abs(loc[1, 2] - 0.5 * h * 1.0) < 1e-15             # right hat x psi_1
    assert abs(loc[1, 3] - 0.5 * h / 3.0) < 1e-15             # right hat x psi_2
    assert abs(loc[0, 3] + 0.5 * h / 3.0) < 1e-15             # left hat x psi_2
    # shared hat at node 1: h0/3 + h1/3
    assert abs(M[idx[0, 1], idx[0, 1]] - (0.4 + 0.9) / 3) < 1e-15
    assert abs(M[idx[0, 1], idx[1, 1]] - 0.9 / 6) < 1e-15


# ---------------------------------------------------------------------------
# Touching pair at high degree, against a closed form in hypergeometric
# functions evaluated with 90 significant digits (mpmath), every entry.
#
# With u = t - x_e in [0, h_e] and v = x_e - s in [0, h_f], the derivative of
# trial function b is a polynomial q_b(v) = sum_j q_bj v^j, and
#   int_0^{h_f} (u + v)^(1-alpha) v^j dv
#     = sum_i C(j, i) (-u)^(j-i) [(u + h_f)^e_i - u^e_i] / e_i,  e_i = 2 - alpha + i
# (v = (u + v) - u, binomial expansion).  Against the test derivative
# g_a(u) = sum_k g_ak u^k the outer integral needs only
#   int_0^{h_e} u^m (u + h_f)^beta du
#     = h_f^beta h_e^(m+1) / (m+1) 2F1(-beta, m+1; m+2; -h_e/h_f)
# and int_0^{h_e} u^(m + e_i) du.  The alternating binomial sums cancel
# heavily, hence the 90 digits.
# ---------------------------------------------------------------------------

def _legendre_power_coeffs(n):
    """Exact power-basis coefficients of L_n (explicit sum formula)."""
    from fractions import Fraction
    c = [Fraction(0)] * (n + 1)
    for k in range(n // 2 + 1):
        c[n - 2 * k] += Fraction((-1) ** k * math.comb(n, k) * math.comb(2 * n - 2 * k, n), 2 ** n)
    return c


def _local_deriv_power_coeffs(P, a):
    """d/dxi of local function a (0: left hat, 1: right hat, 1+p: psi_p)."""
    from fractions import Fraction
    if a == 0:
        return [Fraction(-1, 2)]
    if a == 1:
        return [Fraction(1, 2)]
    p = a - 1
    c = [Fraction(0)] * (p + 2)
    for i, v in enumerate(_legendre_power_coeffs(p - 1)):
        c[i] += v
    for i, v in enumerate(_legendre_power_coeffs(p + 1)):
        c[i] -= v
    return [i * c[i] for i in range(1, len(c))]


def _touch_closed_form(he, hf, P, alpha):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 90
    he, hf, al = mp.mpf(he), mp.mpf(hf), mp.mpf(alpha)

    def in_powers_of(c, s0, s1, scale):
        # scale * sum_k c_k (s0 + s1 y)^k as coefficients of y^j
        out = [mp.mpf(0)] * len(c)
        for k, ck in enumerate(c):
            ck = mp.mpf(ck.numerator) / ck.denominator
            for j in range(k + 1):
                out[j] += ck * mp.binomial(k, j) * s0 ** (k - j) * s1 ** j
        return [scale * x for x in out]

    G = [in_powers_of(_local_deriv_power_coeffs(P, a), mp.mpf(-1), 2 / he, 2 / he)
         for a in range(P + 1)]                       # xi = -1 + 2u/h_e
    Q = [in_powers_of(_local_deriv_power_coeffs(P, b), mp.mpf(1), -2 / hf, 2 / hf)
         for b in range(P + 1)]                       # eta = 1 - 2v/h_f
    cache = {}

    def J(m, beta):
        if (m, beta) not in cache:
            cache[(m, beta)] = (hf ** beta * he ** (m + 1) / (m + 1)
                                * mp.hyp2f1(-beta, m + 1, m + 2, -he / hf))
        return cache[(m, beta)]

    T = [[mp.mpf(0)] * (P + 1) for _ in range(P + 1)]   # T[k][j]
    for k in range(P + 1):
        for j in range(P + 1):
            acc = mp.mpf(0)
            for i in range(j + 1):
                e = 2 - al + i
                m = k + j - i
                acc += (mp.binomial(j, i) * (-1) ** (j - i) / e
                        * (J(m, e) - he ** (m + e + 1) / (m + e + 1)))
            T[k][j] = acc
    g0 = 1 / mp.gamma(2 - al)
    K = np.zeros((P + 1, P + 1))
    for a in range(P + 1):
        for b in range(P + 1):
            acc = mp.mpf(0)
            for k, gk in enumerate(G[a]):
                for j, qj in enumerate(Q[b]):
                    acc += gk * qj * T[k][j]
            K[a, b] = float(g0 * acc)
    return K


@pytest.mark.parametrize("he,hf,alpha", [(0.7, 0.3, 1.3), (0.25, 0.5, 1.05),
                                         (1.0, 1e-3, 1.7), (1e-3, 1.0, 1.95)])
def test_touching_pair_P16_closed_form(he, hf, alpha):
    P = 16
    ref = _touch_closed_form(he, hf, P, alpha)
    got = pair_touch(he, hf, P, alpha)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_touching_pair_closed_form_agrees_with_quadpack():
    """The closed form itself against QUADPACK at low degree (P = 3)."""
    mesh = Mesh(np.array([0.3, 0.7]))
    ref = _touch_closed_form(mesh.h[1], mesh.h[0], 3, 1.35)
    for a, b in [(0, 0), (1, 2), (3, 3), (2, 0)]:
        with warnings.catch_warnings():
            warnings.simplefilter("ignore")
            q = _brute_pair(mesh, 3, 1.35, 1, 0, a, b)
        assert abs(q - ref[a, b]) <= 2e-10 * np.abs(ref).max()
