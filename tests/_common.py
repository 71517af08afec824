"""Helpers shared by the tests: build the same seeded problem for the CUDA
library (through the C ABI binding) and for the oracle."""
import numpy as np

from oracle.basis import Mesh
from paper_1808_02937_gb300 import hfsem as H
from paper_1808_02937_gb300 import workloads as W


def ensure_built():
    import os
    if not os.path.exists(H.LIB_PATH):
        from paper_1808_02937_gb300 import _build
        _build.build()
    return H.load_library()


def gpu_problem(h, P, alpha, theta, rho, a=0.0, b=None, c1=0.0, c2=0.0, matvec=0):
    return H.make_problem(h, P, alpha, theta, rho, a=a, b=b, c1=c1, c2=c2, matvec=matvec)


def oracle_mesh(p):
    return Mesh(p["h"], p["a"], p["b"])


def rel_err(x, y):
    return np.linalg.norm(np.asarray(x) - np.asarray(y)) / max(np.linalg.norm(y), 1e-300)
