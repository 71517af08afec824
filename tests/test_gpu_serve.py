"""The serving loop on the GPU (requests of the config-5 stream: one instance
each, 1..16 right-hand sides, repeated operators):

* every request's solution is the same alone (hfsem_assemble / hfsem_hlu_factor
  / hfsem_solve on its own) and in a mix served by 8 concurrent slots, with
  requests arriving while others run, within 1e-10 relative (the arithmetic
  does not depend on what else runs, so in practice bit for bit);
* the mix reuses resident factorisations and overlaps requests;
* its solutions reproduce the manufactured polynomial solutions where the
  space holds them, and the oracle's discrete solution on the small ones;
* a budget smaller than any request rejects each with HFSEM_ERR_OOM; a budget
  that holds one request at a time serialises them and every one completes.
"""
import time

import numpy as np
import pytest

from oracle.basis import Mesh
from paper_1808_02937_gb300 import hfsem as H
from paper_1808_02937_gb300 import workloads as W
from tests._common import ensure_built, rel_err
from tests._oracle_pool import oracle_solve_many
from tests.test_oracle_solve import expected_coeffs

pytestmark = pytest.mark.gpu

OPTS = dict(R=8, lam=1.0, tol_hlu=1e-3, precision=H.PREC_MIXED)
TOL, MAX_ITER = 1e-14, 100


@pytest.fixture(scope="module")
def lib():
    return ensure_built()


def _requests(n=36, nd_max=4000):
    out = []
    for p in W.config5_requests(600):
        if p.Nd <= nd_max:
            out.append(p)
        if len(out) == n:
            break
    return out


def _alone(p):
    sys_ = H.hfsem_assemble([H.make_problem(p.h, p.P, p.alpha, p.theta, p.rho)])
    fac = H.hfsem_hlu_factor(sys_, H.hopts(**OPTS))
    X, st, code = H.hfsem_solve(sys_, fac, [H.rhs_frac_powers(p.rhs)], tol=TOL,
                                max_iter=MAX_ITER)
    return X.reshape(len(p.rhs), p.Nd).T.copy()


def test_serving_results_same_alone_and_in_mix(lib):
    torch = pytest.importorskip("torch")
    reqs = _requests()
    keys = {(p.N, p.P, p.alpha, p.theta, p.rho, p.h.tobytes()) for p in reqs}
    assert len(keys) < len(reqs)              # some operators repeat
    srv = H.Server(slots=8, cache_factors=64, hopts_=H.hopts(**OPTS), tol=TOL,
                   max_iter=MAX_ITER)
    ids = {}
    half = len(reqs) // 2
    for k, p in enumerate(reqs):
        if k == half:
            time.sleep(0.05)                  # the rest arrive while the first run
        nd = p.Nd * len(p.rhs)
        X = (torch.zeros(nd, dtype=torch.float64, device="cuda") if k % 2
             else np.zeros(nd))               # device and host outputs
        ids[srv.submit(H.make_problem(p.h, p.P, p.alpha, p.theta, p.rho),
                       H.rhs_frac_powers(p.rhs), X=X)] = k
    srv.drain()
    done = {ids[d["id"]]: d for d in srv.poll()}
    c = srv.counters()
    srv.close()
    assert len(done) == len(reqs)
    assert c["builds"] == len(keys) and c["reuses"] == len(reqs) - len(keys)
    assert c["peak_running"] >= 2
    worst = 0.0
    n_exact = 0
    for k, p in enumerate(reqs):
        d = done[k]
        assert d["status"] == H.HFSEM_OK, (p.name, d["msg"], d["stats"])
        X = d["X"].cpu().numpy() if hasattr(d["X"], "cpu") else d["X"]
        mix = X.reshape(len(p.rhs), p.Nd).T
        alone = _alone(p)
        for r in range(len(p.rhs)):
            e = rel_err(mix[:, r], alone[:, r])
            worst = max(worst, e)
            assert e <= 1e-10, (p.name, r, e)
            u = p.u_exact[r]
            if p.P >= len(u) - 1:
                Xe = expected_coeffs(Mesh(p.h, 0.0, 1.0), p.P, np.polynomial.Polynomial(u))
                assert rel_err(mix[:, r], Xe) < 1e-10, (p.name, r)
                n_exact += 1
    print(f"max relative difference alone vs mix: {worst:.3e}; exact reproductions {n_exact}")
    assert n_exact >= 20
    # the oracle's discrete solution on the small requests, first column
    small = [(k, p) for k, p in enumerate(reqs) if p.Nd <= 800][:6]
    ref = oracle_solve_many([(p.h, 0.0, 1.0, p.P, p.alpha, p.theta, p.rho, 0.0, 0.0,
                              ("frac_powers", p.rhs[0])) for _, p in small])
    for (k, p), xo in zip(small, ref):
        X = done[k]["X"]
        X = X.cpu().numpy() if hasattr(X, "cpu") else X
        assert rel_err(X[: p.Nd], xo) < 1e-10, p.name


def test_serving_budget_below_any_request_rejects(lib):
    reqs = _requests(4)
    srv = H.Server(slots=2, budget_bytes=1 << 20, cache_factors=4, hopts_=H.hopts(**OPTS))
    for p in reqs:
        srv.submit(H.make_problem(p.h, p.P, p.alpha, p.theta, p.rho), H.rhs_frac_powers(p.rhs))
    srv.drain()
    done = srv.poll()
    c = srv.counters()
    srv.close()
    assert [d["status"] for d in done] == [H.HFSEM_ERR_OOM] * len(reqs)
    assert c["rejected"] == len(reqs) and c["builds"] == 0


def test_serving_budget_for_one_request_serialises(lib):
    # six distinct operators of one size: measure one request's charge, then
    # give the server room for one at a time only
    base = W.config4(8)
    ps = [p for p in base if p.name.split()[1] == "uniform"][:1] or base[:1]
    p0 = ps[0]
    probs = [H.make_problem(p0.h, p0.P, 1.1 + 0.1 * k, p0.theta, p0.rho) for k in range(6)]
    rhs = H.rhs_frac_powers(p0.rhs[:1])
    srv = H.Server(slots=4, cache_factors=0, hopts_=H.hopts(**OPTS))
    srv.submit(probs[0], rhs)
    srv.drain()
    srv.poll()
    one = srv.counters()["peak_bytes"]
    srv.close()
    srv = H.Server(slots=4, budget_bytes=int(1.5 * one), cache_factors=0, hopts_=H.hopts(**OPTS))
    for pr in probs:
        srv.submit(pr, rhs)
    srv.drain()
    done = srv.poll()
    c = srv.counters()
    srv.close()
    assert all(d["status"] == H.HFSEM_OK for d in done) and len(done) == 6
    assert c["peak_running"] == 1 and c["peak_bytes"] <= int(1.5 * one)
    starts = sorted(d["t_start"] for d in done)
    dones = sorted(d["t_done"] for d in done)
    assert all(s >= e - 1e-9 for s, e in zip(starts[1:], dones[:-1]))
