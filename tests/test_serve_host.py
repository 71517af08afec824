"""Host logic of the serving loop's scheduler (no GPU): the checks live in
tests/serve_check.cpp, which drives the scheduler of csrc/serve_sched.h
with a fake executor that sleeps instead of solving and records, on its own
side, how many requests run at once, the bytes held at any moment and the
order requests start in."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1808_02937_gb300", "csrc")


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no host C++ compiler")
    out = str(tmp_path_factory.mktemp("serve") / "serve_check")
    subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-I", CSRC,
                    os.path.join(HERE, "serve_check.cpp"), "-o", out], check=True)
    return out


def _run(checker, scenario):
    r = subprocess.run([checker, scenario], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    out = {}
    for line in r.stdout.splitlines():
        k, _, v = line.partition(" ")
        out[k] = v
    return out


def _i(d, k):
    return int(d[k])


def _common(d):
    # the budget is never exceeded, by the scheduler's account or the executor's
    assert _i(d, "sched_peak_bytes") <= _i(d, "budget")
    assert _i(d, "exec_peak_held") <= _i(d, "budget")
    assert _i(d, "concurrent_same_key") == 0
    assert _i(d, "live_handles_after_shutdown") == 0


def test_requests_overlap_in_slots(checker):
    d = _run(checker, "overlap")
    _common(d)
    assert _i(d, "exec_peak_running") == 8 and _i(d, "done_ok") == 16


def test_budget_back_pressure(checker):
    d = _run(checker, "backpressure")
    _common(d)
    assert _i(d, "exec_peak_running") == 1 and _i(d, "done_ok") == 6
    assert d["start_order"].split() == [str(i) for i in range(6)]


def test_request_beyond_budget_is_rejected(checker):
    d = _run(checker, "oom")
    _common(d)
    assert _i(d, "done_oom") == 1 and _i(d, "rejected") == 1 and _i(d, "done_ok") == 2
    assert "1" not in d["start_order"].split()


def test_factorisation_reused_exclusively(checker):
    d = _run(checker, "reuse")
    _common(d)
    assert _i(d, "builds") == 1 and _i(d, "reuses") == 4 and _i(d, "done_ok") == 5
    assert _i(d, "exec_peak_running") == 1


def test_idle_factorisations_evicted_least_recent_first(checker):
    d = _run(checker, "evict")
    _common(d)
    assert _i(d, "builds") == 4 and _i(d, "reuses") == 1 and _i(d, "evictions") == 2
    assert d["start_order"].split() == ["0", "1", "2", "3", "4"]


def test_waiting_request_not_overtaken(checker):
    d = _run(checker, "fifo")
    _common(d)
    assert d["start_order"].split() == ["0", "1", "2"]


def test_factorisation_dropped_after_failed_solve(checker):
    d = _run(checker, "drop")
    _common(d)
    # request 0 fails and its factorisation is released; 1 builds anew, 2 reuses it
    assert _i(d, "builds") == 1 and _i(d, "reuses") == 1
    assert _i(d, "done_ok") == 2 and _i(d, "done_oom") == 1
