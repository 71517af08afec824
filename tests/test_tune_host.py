"""The leaf-size table of the autotuner on the host (no GPU): loading a
written table, lookups by class, merging, clearing, and rejection of a
malformed file or NULL arguments.  The timing runs themselves need the GPU
(tests/test_gpu_tune.py)."""
import pytest

from paper_1808_02937_gb300 import hfsem as H
from tests._common import ensure_built


@pytest.fixture()
def lib():
    lib = ensure_built()
    H.hfsem_tune_clear()
    yield lib
    H.hfsem_tune_clear()


def test_load_and_lookup(lib, tmp_path):
    p = tmp_path / "t.txt"
    p.write_text("# comment\n0 1 5 64\n1 1 12 96\n0 0 8 128\n")
    assert H.hfsem_tune_lookup(0, 1, 5) == 0
    H.hfsem_tune_load(str(p))
    assert H.hfsem_tune_lookup(0, 1, 5) == 64
    assert H.hfsem_tune_lookup(1, 1, 12) == 96
    assert H.hfsem_tune_lookup(0, 0, 8) == 128
    assert H.hfsem_tune_lookup(0, 0, 5) == 0          # no entry for that class
    assert H.hfsem_tune_lookup(1, 1, 5) == 0
    # a second file merges (and overrides) entries
    q = tmp_path / "u.txt"
    q.write_text("0 1 5 48\n0 1 6 32\n")
    H.hfsem_tune_load(str(q))
    assert H.hfsem_tune_lookup(0, 1, 5) == 48
    assert H.hfsem_tune_lookup(0, 1, 6) == 32
    assert H.hfsem_tune_lookup(1, 1, 12) == 96
    H.hfsem_tune_clear()
    assert H.hfsem_tune_lookup(0, 1, 5) == 0


@pytest.mark.parametrize("bad", ["0 1 5\n", "2 1 5 64\n", "0 1 0 64\n", "0 1 5 0\n",
                                 "0 1 5 129\n", "x y z w\n", "0 2 5 64\n"])
def test_malformed_table_is_rejected_whole(lib, tmp_path, bad):
    p = tmp_path / "t.txt"
    p.write_text("0 1 7 64\n" + bad)
    with pytest.raises(H.HfsemError) as e:
        H.hfsem_tune_load(str(p))
    assert e.value.code == H.HFSEM_ERR_INVALID_ARG
    assert H.hfsem_tune_lookup(0, 1, 7) == 0          # nothing of it entered the table


def test_null_arguments(lib, tmp_path):
    assert lib.hfsem_tune_load(None) == H.HFSEM_ERR_INVALID_ARG
    assert lib.hfsem_tune_load(str(tmp_path / "missing.txt").encode()) == H.HFSEM_ERR_INVALID_ARG
    assert lib.hfsem_tune_lookup(0, 1, 5, None) == H.HFSEM_ERR_INVALID_ARG
    assert lib.hfsem_tune(None, None, None, 1e-14, 10, None, None, 0, None) == H.HFSEM_ERR_INVALID_ARG
