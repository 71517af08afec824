"""Pins for the oracle's load vector of a Legendre-series right-hand side
(Sec. 2.2, G_i = (f, phi_i)), f = sum_k g_k L_k(xi_[a,b](x)).

The expected values are exact polynomial integrals formed with numpy's own
Legendre-series arithmetic, not with the oracle's quadrature or recurrence:
on element e the series is re-expanded on the element's reference
coordinate (numpy's domain conversion), multiplied by the local basis
function written as a Legendre series (hats (1 -+ xi)/2, bubbles
L_{p-1} - L_{p+1}) and integrated as 2 c_0 times the Jacobian h_e / 2.
Meshes are graded and the interval does not start at 0, so a wrong map of
[a, b] onto [-1, 1] or a rule one point short of exact shows up."""
import numpy as np
import numpy.polynomial.legendre as npleg
import pytest
from numpy.polynomial import Legendre

import oracle.load as OL
from oracle.basis import Mesh
from paper_1808_02937_gb300 import workloads as W


def _basis_series(P):
    """Local basis as Legendre coefficient vectors: left hat, right hat,
    bubbles psi_p = L_{p-1} - L_{p+1}."""
    out = [np.array([0.5, -0.5]), np.array([0.5, 0.5])]
    for p in range(1, P):
        c = np.zeros(p + 2)
        c[p - 1] += 1.0
        c[p + 1] -= 1.0
        out.append(c)
    return out


def _exact_load(h, a, b, P, g):
    """Exact G in X's ordering followed by the boundary hats at a and at b."""
    N = len(h)
    nodes = a + np.concatenate([[0.0], np.cumsum(h)])
    nodes[-1] = b
    f = Legendre(g, domain=[a, b])
    basis = _basis_series(P)
    Nd = N * P - 1
    G = np.zeros(Nd + 2)
    for e in range(N):
        fe = f.convert(domain=[nodes[e], nodes[e + 1]]).coef   # series in xi
        vals = [h[e] * npleg.legmul(fe, c)[0] for c in basis]    # (h/2) * 2 c_0
        left = Nd if e == 0 else N * (P - 1) + e - 1
        right = Nd + 1 if e == N - 1 else N * (P - 1) + e
        G[left] += vals[0]
        G[right] += vals[1]
        for p in range(1, P):
            G[e * (P - 1) + p - 1] += vals[1 + p]
    return G


CASES = [
    # (mesh lengths, a, P, K)
    (W.mesh_graded(7, 2.0, 0.0, 2.0), -0.3, 4, 9),
    (W.mesh_graded(5, 3.0, 0.0, 1.5), 0.4, 16, 32),
    (W.mesh_geometric_two_sided(8, 0.5, 0.0, 1.0), 2.0, 8, 32),
    (W.mesh_uniform(3, 0.0, 0.7), -1.1, 1, 5),
    (np.array([1.3]), 0.25, 6, 0),
]


def _case(k):
    h, a, P, K = CASES[k]
    g = np.random.default_rng(100 + k).standard_normal(K + 1)
    b = a + float(h.sum())
    return h, a, b, P, g


@pytest.mark.parametrize("k", range(len(CASES)))
def test_legendre_load_exact_polynomial_integrals(k):
    h, a, b, P, g = _case(k)
    got = OL.load_legendre_ab(Mesh(h, a, b), P, g)
    ref = _exact_load(h, a, b, P, g)
    # exact up to rounding: measured 5e-16 .. 2.7e-15 of the largest entry
    assert np.abs(got - ref).max() <= 2e-14 * np.abs(ref).max()


def test_legendre_load_pin_catches_planted_mistakes(monkeypatch):
    """The pin above fails when the oracle's rule loses one point or the map
    of [a, b] onto [-1, 1] is shifted (mistakes planted in the oracle)."""
    h, a, b, P, g = _case(1)
    g = np.zeros_like(g)
    g[-1] = 1.0                    # f = L_32: the top degree decides exactness
    ref = _exact_load(h, a, b, P, g)
    bar = 2e-14 * np.abs(ref).max()

    real_gl = OL.gauss_legendre
    monkeypatch.setattr(OL, "gauss_legendre", lambda n: real_gl(n - 1))
    short = OL.load_legendre_ab(Mesh(h, a, b), P, g)
    assert np.abs(short - ref).max() > 100 * bar
    monkeypatch.setattr(OL, "gauss_legendre", real_gl)

    real_leg = OL.legendre_all
    monkeypatch.setattr(OL, "legendre_all", lambda K, t: real_leg(K, t + 1e-3))
    shifted = OL.load_legendre_ab(Mesh(h, a, b), P, g)
    assert np.abs(shifted - ref).max() > 100 * bar
