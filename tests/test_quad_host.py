"""Host-side Gauss-Jacobi rules of the CUDA path (csrc/quad_host.cpp: Sturm
bisection for the nodes, Christoffel weights), compiled here with the host
compiler: nodes and weights against scipy's Golub-Welsch rules, and exact
moments of the weight (1-x)^a (1+x)^b for every degree up to 2n-1 against the
Beta-function closed form, including the fractional exponents of the singular
pair integrals (-1 < a, b < 1)."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest
from scipy import special

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1808_02937_gb300", "csrc")

CASES = [(1, 0.0, 0.0), (5, 0.0, 0.0), (12, 0.0, 0.0), (30, 0.0, 0.0),
         (8, -0.5, -0.5), (10, 0.3, -0.6), (16, -0.4, 0.0), (20, 0.0, 0.7),
         (24, -0.2, 0.8), (7, 0.9, -0.9), (9, -0.7, -0.3 + 1e-9)]


@pytest.fixture(scope="module")
def rules(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path_factory.mktemp("quad") / "quad_check")
    inc = ["-I", CSRC, "-I", os.path.join(ROOT, "include")]
    if os.path.isdir("/usr/local/cuda/include"):
        inc += ["-I", "/usr/local/cuda/include"]
    subprocess.run([cxx, "-O2", "-std=c++17", *inc, os.path.join(HERE, "quad_check.cpp"),
                    os.path.join(CSRC, "quad_host.cpp"), "-o", exe], check=True)
    inp = "".join(f"{n} {a!r} {b!r}\n" for n, a, b in CASES)
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    vals = np.array([[float(t) for t in line.split()] for line in out.strip().splitlines()])
    res, k = {}, 0
    for n, a, b in CASES:
        res[(n, a, b)] = (vals[k:k + n, 0], vals[k:k + n, 1])
        k += n
    return res


def _moment(k, a, b):
    # int_{-1}^{1} (1-x)^a (1+x)^b x^k dx with x = 2t - 1:
    # 2^(a+b+1) sum_j C(k,j) 2^j (-1)^(k-j) B(b+j+1, a+1)
    s = 0.0
    for j in range(k + 1):
        s += math.comb(k, j) * 2.0 ** j * (-1.0) ** (k - j) * special.beta(b + j + 1, a + 1)
    return 2.0 ** (a + b + 1) * s


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}_a{c[1]}_b{c[2]}")
def test_rule_matches_golub_welsch(rules, case):
    n, a, b = case
    x, w = rules[case]
    xr, wr = special.roots_jacobi(n, a, b)
    assert np.all(np.diff(x) > 0) and np.all(np.abs(x) < 1) and np.all(w > 0)
    assert np.max(np.abs(x - xr)) < 1e-14
    assert np.max(np.abs(w - wr) / wr) < 1e-12


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"n{c[0]}_a{c[1]}_b{c[2]}")
def test_rule_is_exact_to_degree_2n_minus_1(rules, case):
    n, a, b = case
    x, w = rules[case]
    for k in range(0, min(2 * n, 16)):
        m = _moment(k, a, b)
        scale = 2.0 ** (a + b + 1) * special.beta(b + 1, a + 1)   # the zeroth moment
        assert abs(np.dot(w, x ** k) - m) < 1e-13 * scale * 2 ** k, (k, np.dot(w, x ** k), m)
