"""The leaf-size autotuner on the GPU (Sec. 4.1 leaves the cluster tree's
leaf size open): it times every candidate per instance class, its choice is
what a later factorisation with leaf_elems = 0 uses (the same solution and
iterations as the explicit size), the chosen size is never slower than the
automatic one among the sizes with the fewest iterations, and the written
table reloads."""
import numpy as np
import pytest

from paper_1808_02937_gb300 import hfsem as H
from paper_1808_02937_gb300 import workloads as W
from tests._common import ensure_built

pytestmark = pytest.mark.gpu


@pytest.fixture()
def lib():
    lib = ensure_built()
    H.hfsem_tune_clear()
    yield lib
    H.hfsem_tune_clear()


def _opts(leaf=0):
    return H.hopts(R=8, lam=1.0, tol_hlu=1e-3, precision=H.PREC_MIXED, leaf_elems=leaf,
                   admissibility=H.ADM_MIN)


def test_tuned_leaf_is_used_and_reloads(lib, tmp_path):
    insts = [p for p in W.config4() if p.P == 5 and "uniform" in p.name][:6]
    assert len(insts) >= 3
    probs = [H.make_problem(p.h, p.P, p.alpha, p.theta, p.rho) for p in insts]
    rhs = [H.rhs_frac_powers(p.rhs) for p in insts]
    sys_ = H.hfsem_assemble(probs)
    path = str(tmp_path / "leaf.txt")
    got = H.hfsem_tune(sys_, _opts(), rhs, tol=1e-14, max_iter=100, path=path)
    assert len(got) == 1
    e = got[0]
    assert (e["fp64"], e["kind"], e["P"]) == (0, 0, 5) and e["n_inst"] == 32
    assert e["leaf_dofs"] in (32, 48, 64, 96, 128)
    assert e["ms"] > 0 and e["ms_default"] > 0
    assert H.hfsem_tune_lookup(0, 0, 5) == e["leaf_dofs"]
    # leaf_elems = 0 now means the tuned size
    f0 = H.hfsem_hlu_factor(sys_, _opts())
    X0, s0, c0 = H.hfsem_solve(sys_, f0, rhs, tol=1e-14, max_iter=100)
    f1 = H.hfsem_hlu_factor(sys_, _opts(max(1, e["leaf_dofs"] // 5)))
    X1, s1, c1 = H.hfsem_solve(sys_, f1, rhs, tol=1e-14, max_iter=100)
    assert c0 == c1 == H.HFSEM_OK
    assert [s["iters"] for s in s0] == [s["iters"] for s in s1]
    assert np.array_equal(X0, X1)
    # the file holds the table; it reloads into a cleared one
    assert "0 0 5 %d" % e["leaf_dofs"] in open(path).read()
    H.hfsem_tune_clear()
    assert H.hfsem_tune_lookup(0, 0, 5) == 0
    H.hfsem_tune_load(path)
    assert H.hfsem_tune_lookup(0, 0, 5) == e["leaf_dofs"]


def test_tune_over_classes(lib):
    # several classes in one batch (uniform / graded / geometric, a few P)
    insts = [p for p in W.config4()[:80] if p.P in (3, 8)][:16]
    probs = [H.make_problem(p.h, p.P, p.alpha, p.theta, p.rho,
                            matvec=H.MATVEC_AUTO if np.ptp(p.h) <= 1e-13 * p.h.max()
                            else H.MATVEC_HMATRIX) for p in insts]
    rhs = [H.rhs_frac_powers(p.rhs) for p in insts]
    sys_ = H.hfsem_assemble(probs)
    got = H.hfsem_tune(sys_, _opts(), rhs, tol=1e-14, max_iter=100)
    classes = {(int(p.h.max() > 1e45 * p.h.min()), int(np.ptp(p.h) > 1e-13 * p.h.max()), p.P)
               for p in insts}
    assert {(e["fp64"], e["kind"], e["P"]) for e in got} == classes
    for e in got:
        assert H.hfsem_tune_lookup(e["fp64"], e["kind"], e["P"]) == e["leaf_dofs"]
        assert e["leaf_dofs"] <= (96 if e["fp64"] else 128)
    # the batch factors and solves with the tuned sizes
    fac = H.hfsem_hlu_factor(sys_, _opts())
    X, st, code = H.hfsem_solve(sys_, fac, rhs, tol=1e-14, max_iter=100)
    assert code == H.HFSEM_OK
