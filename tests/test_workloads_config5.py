"""The seeded request stream (config 5) and its largest request: shapes,
ranges, determinism and the share of repeated factor keys."""
import math

import numpy as np

from paper_1808_02937_gb300 import workloads as W


def test_stream_shapes_and_ranges():
    reqs = list(W.config5_requests(600))
    assert len(reqs) == 600
    for p in reqs:
        assert 1 <= p.N <= 4096 and 2 <= p.P <= 16
        assert 1 <= len(p.rhs) <= 16 and len(p.u_exact) == len(p.rhs)
        assert np.all(p.h > 0.0) and abs(p.h.sum() - 1.0) < 1e-12
        assert 1.1 <= p.alpha <= 1.9 and 0.0 <= p.theta <= 1.0 and 0.0 <= p.rho <= 2.0
        for u in p.u_exact:
            assert len(u) - 1 <= 6 and u[0] == 0.0 and abs(np.polyval(u[::-1], 1.0)) < 1e-12
    nd = np.array([p.Nd for p in reqs])
    assert nd.min() >= 99 and nd.max() <= 65535
    # log-uniform sizes: the median sits near the geometric mean of the range
    assert 1000 < np.median(nd) < 8000


def test_stream_reuse_and_arrivals():
    reqs = list(W.config5_requests(2000, rate=5.0))
    reuse = [p for p in reqs if p.reuse_of >= 0]
    assert 0.25 < len(reuse) / len(reqs) < 0.35
    for p in reuse[:50]:
        q = reqs[p.reuse_of]
        assert q.reuse_of == -1
        assert (p.N, p.P, p.alpha, p.theta, p.rho) == (q.N, q.P, q.alpha, q.theta, q.rho)
        assert np.array_equal(p.h, q.h)
    t = np.array([p.arrival for p in reqs])
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 0.2) < 0.02


def test_stream_is_seeded():
    a = [p.name for p in W.config5_requests(40)]
    b = [p.name for p in W.config5_requests(40)]
    c = [p.name for p in W.config5_requests(40, seed=7)]
    assert a == b and a != c


def test_geometric_floor_keeps_meshes_representable():
    for N in (256, 1024, 4096):
        q = W.geometric_q_floor(N)
        h = W.mesh_geometric_two_sided(N, q)
        assert h.min() > 0.0 and h.min() / h.max() > 1e-300
        assert q ** (N // 2 - 1) >= 1e-281 and math.isfinite(q)


def test_largest_request():
    for fam in ("uniform", "graded"):
        p = W.config5_max_request(fam)
        assert (p.N, p.P, p.Nd, len(p.rhs)) == (4096, 16, 65535, 16)
        assert np.all(p.h > 0.0) and abs(p.h.sum() - 1.0) < 1e-12
