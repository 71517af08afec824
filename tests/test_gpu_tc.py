"""The tensor-core mode of the H-LU (dense leaf products on tcgen05 with
each FP32 operand split into a BF16 head and a BF16 tail, three MMAs per K
step, FP32 accumulation in tensor memory):

* the tile on its own, every entry within the error bound of the split
  (the dropped tail-tail product and the two roundings, about 2^-16
  relative) plus FP32 accumulation, with several products per CTA on one
  completion barrier;
* a full-size factorisation and solve (nine uniform instances, N = 1024,
  P = 8) in that mode: as strong a preconditioner as the FP32 mode (at most
  one more iteration per column), and the FP64 Krylov loop reaches the
  oracle's solution.
"""
import numpy as np
import pytest

from oracle.basis import Mesh
from oracle.solve import solve_problem
from paper_1808_02937_gb300 import hfsem as H
from paper_1808_02937_gb300 import workloads as W
from tests._common import ensure_built, rel_err
from tests._oracle_pool import config2_oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    return ensure_built()


@pytest.mark.parametrize("N,K,reps", [(16, 64, 1), (32, 128, 3), (48, 80, 2), (128, 128, 4)])
def test_tc_tile_within_split_bound(lib, N, K, reps):
    err = H.hfsem_tc_tile_check(N, K, reps)
    # a = a_h + a_l + d_a with |d_a| <= u^2 |a| (u = 2^-9, BF16 nearest, two
    # roundings); a_h b_h + a_h b_l + a_l b_h misses a_l b_l (<= u^2 |ab|) and
    # the d terms (<= 2 u^2 (1 + u) |ab|): <= 4 u^2 |ab| = 2^-16 |ab|, plus
    # FP32 accumulation over 3K terms
    bound = 2.0 ** -16 + 3 * K * 2.0 ** -24
    # plain BF16 operands would give up to 2^-8: the split must do far better
    assert bound < 2.0 ** -12
    assert 0.0 <= err <= bound, (err, bound)


def test_tc_tile_bad_arguments(lib):
    for N, K in ((8, 64), (24, 64), (32, 48), (32, 136)):
        with pytest.raises(H.HfsemError) as ei:
            H.hfsem_tc_tile_check(N, K, 1)
        assert ei.value.code == H.HFSEM_ERR_INVALID_ARG


def test_mixed_tc_config2_reaches_oracle(lib):
    insts = W.config2()
    ref = config2_oracle()
    sys_ = H.hfsem_assemble([H.make_problem(p.h, p.P, p.alpha, p.theta, p.rho) for p in insts])
    rhs = [H.rhs_legendre([p.rhs[0]]) for p in insts]
    f32 = H.hfsem_hlu_factor(sys_, H.hopts(R=8, lam=1.0, tol_hlu=1e-3, precision=H.PREC_MIXED))
    _, s32, _ = H.hfsem_solve(sys_, f32, rhs, tol=1e-14, max_iter=80)
    fac = H.hfsem_hlu_factor(sys_, H.hopts(R=8, lam=1.0, tol_hlu=1e-3,
                                           precision=H.PREC_MIXED_TC))
    X, st, code = H.hfsem_solve(sys_, fac, rhs, tol=1e-14, max_iter=80)
    assert code == H.HFSEM_OK, st
    for s, s_ref in zip(st, s32):
        # as strong as the FP32 preconditioner: at most one more iteration;
        # accepted on the true residual (<= 100 tol, or at the FP64 floor)
        assert s["iters"] <= s_ref["iters"] + 1, (st, s32)
        assert s["rel_true_residual"] < 1e-11, st
    parts = H.split(sys_, X)
    for k in range(len(insts)):
        assert rel_err(parts[k][:, 0], ref[k]) < 1e-10, k
