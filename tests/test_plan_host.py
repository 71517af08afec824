"""Host logic of the H-LU planner (no GPU): the block tree covers the matrix
exactly once with admissible low-rank blocks (Sec. 3.1), the ops of each
wave of the H-LU program touch disjoint storage (the CTAs of a cluster run
them concurrently), and the leaf-solve tables stay in bounds.  The checks
live in tests/plan_check.cpp, compiled here against the planner source with
the host compiler; they share no code with the planner's own dependency
analysis."""
import os
import shutil
import subprocess

import pytest

from paper_1808_02937_gb300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1808_02937_gb300", "csrc")


@pytest.fixture(scope="module")
def verifier(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("plan") / "plan_check")
    inc = ["-I", CSRC, "-I", os.path.join(ROOT, "include")]
    cuda_inc = "/usr/local/cuda/include"
    if os.path.isdir(cuda_inc):
        inc += ["-I", cuda_inc]
    subprocess.run([cxx, "-O2", "-std=c++17", *inc, os.path.join(HERE, "plan_check.cpp"),
                    os.path.join(CSRC, "hmatrix_plan.cpp"), "-o", out], check=True)
    return out


def _run(verifier, h, P, leaf, R, lam=1.0, mode=0, rule=0):
    inp = (f"{len(h)} {P} {leaf} {R} {lam} {mode} {rule}\n" +
           " ".join(repr(float(v)) for v in h) + "\n")
    return subprocess.run([verifier], input=inp, capture_output=True, text=True, timeout=300)


CASES = [
    ("uniform", W.mesh_uniform(48), 4, 4, 4),
    ("graded3", W.mesh_graded(40, 3.0), 3, 2, 5),
    ("geo2", W.mesh_geometric_two_sided(32, 0.5), 5, 2, 6),
    ("ragged", W.mesh_graded(19, 2.0), 2, 2, 3),
    ("uniform-N256-P8", W.mesh_uniform(256), 8, 16, 8),
    ("graded-N200-P6", W.mesh_graded(200, 2.0), 6, 16, 8),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: c[0])
@pytest.mark.parametrize("rule", [0, 1], ids=["adm-max", "adm-min"])
def test_plan_is_race_free_and_in_bounds(verifier, case, rule):
    name, h, P, leaf, R = case
    r = _run(verifier, h, P, leaf, R, rule=rule)
    assert r.returncode == 0 and r.stdout.startswith("OK"), (r.stdout, r.stderr)


def test_min_admissibility_on_geometric_mesh(verifier):
    # an extreme two-sided geometric mesh (elements from 1 down to ~1e-60)
    h = W.mesh_geometric_two_sided(200, 0.25)
    r = _run(verifier, h, 3, 8, 6, rule=1)
    assert r.returncode == 0 and r.stdout.startswith("OK"), (r.stdout, r.stderr)


def test_verifier_sees_conflicts(verifier):
    # the whole H-LU program as one wave must conflict: the factorisation is a
    # chain of dependent ops, so a verifier that passes this is not looking
    h = W.mesh_uniform(48)
    r = _run(verifier, h, 4, 4, 4, mode=1)
    assert r.returncode != 0 and r.stdout.startswith("FAIL"), r.stdout
    assert "wave" in r.stdout
