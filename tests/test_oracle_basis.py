"""Pins for the reference basis (Sec. 2.2) against numpy's Legendre module
and the properties the paper states."""
import numpy as np
import numpy.polynomial.legendre as npleg

from oracle.basis import (Mesh, global_index, legendre_all, legendre_deriv_all,
                          local_derivs, local_values, n_dof)
from oracle.quadrature import gauss_legendre


def test_legendre_matches_numpy():
    x = np.linspace(-1, 1, 37)
    L = legendre_all(12, x)
    dL = legendre_deriv_all(12, x)
    for p in range(13):
        c = np.zeros(p + 1)
        c[p] = 1
        assert np.allclose(L[p], npleg.legval(x, c), atol=1e-14)
        assert np.allclose(dL[p], npleg.legval(x, npleg.legder(c)), atol=1e-12)


def test_orthogonality_and_endpoints():
    # int L_p L_q = 2/(2p+1) delta_pq and L_p(+-1) = (+-1)^p (Sec. 2.2)
    x, w = gauss_legendre(20)
    L = legendre_all(10, x)
    G = (L * w) @ L.T
    assert np.allclose(G, np.diag(2.0 / (2 * np.arange(11) + 1)), atol=1e-14)
    ends = legendre_all(10, np.array([-1.0, 1.0]))
    assert np.allclose(ends[:, 0], (-1.0) ** np.arange(11))
    assert np.allclose(ends[:, 1], 1.0)


def test_bubbles_vanish_and_derivative_identity():
    # psi_p(+-1) = 0 (eq. (RefBasis)); psi_p' = -(2p+1) L_p (Legendre identity)
    P = 9
    V = local_values(P, np.array([-1.0, 1.0]))
    assert np.allclose(V[2:], 0.0, atol=1e-14)
    x = np.linspace(-1, 1, 11)
    D = local_derivs(P, x)
    L = legendre_all(P, x)
    for p in range(1, P):
        assert np.allclose(D[1 + p], -(2 * p + 1) * L[p], atol=1e-12)
    assert np.allclose(D[0], -0.5) and np.allclose(D[1], 0.5)


def test_ordering_and_count():
    # X = [bubbles element by element; interior hats], N_d = N P - 1
    N, P = 5, 4
    idx = global_index(N, P)
    Nd = n_dof(N, P)
    assert Nd == N * P - 1
    assert idx[0, 0] == Nd and idx[N - 1, 1] == Nd + 1
    assert sorted(set(idx.ravel().tolist())) == list(range(Nd + 2))
    assert idx[2, 1 + 1] == 2 * (P - 1)          # first bubble of element 2
    assert idx[0, 1] == N * (P - 1)              # hat at node 1


def test_mesh_distances_survive_extreme_refinement():
    h = np.array([0.5, 0.25, 2.0 ** -129, 2.0 ** -129])
    m = Mesh(h, 0.0)
    assert m.gap(2, 3) == 0.0
    assert m.node_diff(4, 3) == 2.0 ** -129      # from the right end
    assert m.gap(1, 3) == 2.0 ** -129
