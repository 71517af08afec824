"""The spawn-started oracle worker pool the GPU parity tests use returns the
same solutions as an in-process oracle call (host logic, no GPU)."""
import numpy as np
import pytest

from oracle.basis import Mesh
from oracle.solve import solve_problem
from paper_1808_02937_gb300 import workloads as W
from tests._oracle_pool import oracle_solve_many


@pytest.mark.timeout(300)
def test_pool_matches_in_process_oracle():
    p = W.config1()
    q = W.config2()[0]
    jobs = [(p.h, 0.0, 1.0, p.P, p.alpha, p.theta, p.rho, 0.3, -0.2, ("frac_powers", p.rhs[0])),
            (W.mesh_graded(12, 2.0), 0.0, 1.0, 5, 1.7, 0.2, 0.5, 0.0, 0.0,
             ("legendre_ab", q.rhs[0][:9]))]
    got = oracle_solve_many(jobs)
    for job, x in zip(jobs, got):
        h, a, b, P, alpha, theta, rho, c1, c2, rhs = job
        ref, _ = solve_problem(Mesh(h, a, b), P, alpha, theta, rho, c1, c2, rhs)
        assert np.array_equal(x, ref)
