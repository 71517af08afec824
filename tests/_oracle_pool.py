"""Oracle solves run in worker processes started with 'spawn' (a process
forked after CUDA has been initialised can hang).  Inputs are passed as plain
Python lists, so that a worker sets its BLAS thread count before numpy loads.
Results are cached for the test session under a caller-chosen key."""
import multiprocessing as mp
import os

_cache = {}


def _init(threads):
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = str(threads)


def _solve(job):
    import numpy as np

    from oracle.basis import Mesh
    from oracle.solve import solve_problem
    h, a, b, P, alpha, theta, rho, c1, c2, (kind, data) = job
    if kind == "frac_powers":
        data = [tuple(t) for t in data]
    else:
        data = np.asarray(data, dtype=np.float64)
    X, _ = solve_problem(Mesh(np.asarray(h), a, b), P, alpha, theta, rho, c1, c2, (kind, data))
    return X.tolist()


def _plain(x):
    if hasattr(x, "tolist"):
        return x.tolist()
    if isinstance(x, (list, tuple)):
        return [_plain(v) for v in x]
    return x


def oracle_solve_many(jobs, key=None):
    """jobs: (h, a, b, P, alpha, theta, rho, c1, c2, (kind, data)) tuples;
    returns the oracle's solutions (numpy arrays) in order."""
    import numpy as np
    if key is not None and key in _cache:
        return _cache[key]
    jobs = [tuple(_plain(v) for v in j[:9]) + ((j[9][0], _plain(j[9][1])),) for j in jobs]
    cores = os.cpu_count() or 2
    n = max(1, min(len(jobs), cores // 2))
    ctx = mp.get_context("spawn")
    with ctx.Pool(n, initializer=_init, initargs=(max(1, cores // n),)) as pool:
        out = [np.asarray(x) for x in pool.map(_solve, jobs)]
    if key is not None:
        _cache[key] = out
    return out


def config2_oracle():
    """Oracle solutions of the nine config-2 instances (uniform N = 1024,
    P = 8, Legendre right-hand sides)."""
    from paper_1808_02937_gb300 import workloads as W
    jobs = [(p.h, 0.0, 1.0, p.P, p.alpha, p.theta, p.rho, 0.0, 0.0, ("legendre_ab", p.rhs[0]))
            for p in W.config2()]
    return oracle_solve_many(jobs, key="config2")
