"""hfsem_apply_noalloc: the operator product for callers that cannot
allocate device memory during the call (they own every allocation, or run in
a section where cudaMalloc is not allowed).  Its output must match
hfsem_apply's, call after call, although every call reuses the same
library-held scratch array.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_1808_02937_gb300 import hfsem as H
from paper_1808_02937_gb300 import workloads as W
from tests._common import ensure_built

pytestmark = pytest.mark.gpu


def _system():
    # one Toeplitz (uniform) and one dense (graded) instance: both paths
    return H.hfsem_assemble([
        H.make_problem(W.mesh_uniform(96), 6, 1.5, 0.3, 1.0),
        H.make_problem(W.mesh_graded(40, 3.0), 5, 1.7, 0.8, 0.5),
    ])


def test_noalloc_matches_apply_twice():
    torch = pytest.importorskip("torch")
    ensure_built()
    sys_ = _system()
    rng = np.random.default_rng(17)
    for call in range(2):      # two calls in a row: no state carried over
        nrhs = 1 + call
        x = torch.tensor(rng.standard_normal(sys_.total_ndof * nrhs), device="cuda")
        ref = H.hfsem_apply(sys_, x, nrhs=nrhs).cpu().numpy()
        got = H.hfsem_apply_noalloc(sys_, x, nrhs=nrhs).cpu().numpy()
        scale = np.abs(ref).max()
        assert np.abs(got - ref).max() <= 5e-13 * scale, call


def test_noalloc_leaves_free_memory_unchanged():
    """After the system exists, a call reserves no device memory, the first
    one included (hfsem_assemble loaded the scratch array and the kernels)."""
    torch = pytest.importorskip("torch")
    ensure_built()
    sys_ = _system()
    x = torch.tensor(np.random.default_rng(5).standard_normal(sys_.total_ndof), device="cuda")
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    for call in range(2):
        free0 = torch.cuda.mem_get_info()[0]
        H.hfsem_apply_noalloc(sys_, x, nrhs=1, out=y)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0, call


def test_noalloc_rejects_oversized_requests():
    torch = pytest.importorskip("torch")
    ensure_built()
    sys_ = H.hfsem_assemble([H.make_problem(W.mesh_uniform(1024), 8, 1.5, 0.3, 1.0)])
    x = torch.zeros(sys_.total_ndof * 64, dtype=torch.float64, device="cuda")
    with pytest.raises(H.HfsemError) as e:
        H.hfsem_apply_noalloc(sys_, x, nrhs=64)
    assert e.value.code == H.HFSEM_ERR_INVALID_ARG
    # host pointers are refused as well
    with pytest.raises(H.HfsemError):
        H.hfsem_apply_noalloc(sys_, np.zeros(sys_.total_ndof), nrhs=1)
