"""Argument checking at the C-ABI boundary (no GPU needed: every call below is
rejected before the library touches CUDA).  Each entry point returns
HFSEM_ERR_INVALID_ARG for out-of-range parameters and NULL handles, never
throws across the boundary, and leaves its outputs unwritten."""
import ctypes as C

import numpy as np
import pytest

from paper_1808_02937_gb300 import hfsem as H
from tests._common import ensure_built


@pytest.fixture(scope="module")
def lib():
    return ensure_built()


def _problem(**kw):
    h = np.full(8, 1.0 / 8)
    p = dict(n_elem=8, P=4, a=0.0, b=1.0, h=h, alpha=1.5, theta=0.5, rho=1.0, c1=0.0, c2=0.0,
             matvec=0)
    p.update(kw)
    hh = p["h"]
    ptr = None if hh is None else np.ascontiguousarray(hh).ctypes.data_as(C.POINTER(C.c_double))
    prob = H.hfsem_problem(p["n_elem"], p["P"], p["a"], p["b"], ptr, p["alpha"], p["theta"],
                           p["rho"], p["c1"], p["c2"], p["matvec"])
    return prob, hh


BAD = [
    dict(alpha=1.0), dict(alpha=2.0), dict(alpha=float("nan")),
    dict(theta=-0.1), dict(theta=1.1),
    dict(rho=-1.0), dict(rho=float("inf")),
    dict(P=0), dict(P=33),
    dict(n_elem=0),
    dict(matvec=4), dict(matvec=-1),
    dict(h=None),
    dict(h=np.array([0.5, 0.5, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0])),      # zero lengths
    dict(h=np.full(8, 0.2)),                                           # sum(h) != b - a
    dict(a=1.0, b=0.0, h=np.full(8, -1.0 / 8)),                        # a >= b
    dict(matvec=7),
    dict(c1=float("inf")),
]


@pytest.mark.parametrize("bad", BAD, ids=lambda d: ",".join(f"{k}" for k in d))
def test_assemble_rejects(lib, bad):
    prob, keep = _problem(**bad)
    arr = (H.hfsem_problem * 1)(prob)
    out = C.c_void_p(None)
    code = lib.hfsem_assemble(1, arr, None, C.byref(out))
    assert code == H.HFSEM_ERR_INVALID_ARG
    assert out.value is None


def test_assemble_rejects_empty_batch(lib):
    out = C.c_void_p(None)
    assert lib.hfsem_assemble(0, None, None, C.byref(out)) == H.HFSEM_ERR_INVALID_ARG
    prob, keep = _problem()
    arr = (H.hfsem_problem * 1)(prob)
    assert lib.hfsem_assemble(-1, arr, None, C.byref(out)) == H.HFSEM_ERR_INVALID_ARG
    assert out.value is None


def test_one_bad_instance_rejects_the_batch(lib):
    good, k1 = _problem()
    bad, k2 = _problem(theta=2.0)
    arr = (H.hfsem_problem * 2)(good, bad)
    out = C.c_void_p(None)
    assert lib.hfsem_assemble(2, arr, None, C.byref(out)) == H.HFSEM_ERR_INVALID_ARG
    assert out.value is None


def test_null_handles(lib):
    x = np.zeros(16)
    px = x.ctypes.data_as(C.c_void_p)
    nd = C.c_int32(-7)
    assert lib.hfsem_ndof(None, 0, C.byref(nd)) == H.HFSEM_ERR_INVALID_ARG and nd.value == -7
    assert lib.hfsem_apply(None, 1, px, px) == H.HFSEM_ERR_INVALID_ARG
    assert lib.hfsem_apply_noalloc(None, 1, px, px) == H.HFSEM_ERR_INVALID_ARG
    assert lib.hfsem_load_vector(None, None, 0, px) == H.HFSEM_ERR_INVALID_ARG
    opts = H.hopts()
    fac = C.c_void_p(None)
    assert lib.hfsem_hlu_factor(None, C.byref(opts), C.byref(fac)) == H.HFSEM_ERR_INVALID_ARG
    assert fac.value is None
    assert lib.hfsem_hmatrix_dense(None, 0, px) == H.HFSEM_ERR_INVALID_ARG
    assert lib.hfsem_precond_apply(None, 1, px, px) == H.HFSEM_ERR_INVALID_ARG
    stats = (H.hfsem_stats * 1)()
    rhs = (H.hfsem_rhs * 1)()
    assert lib.hfsem_solve(None, None, rhs, 1e-12, 10, px, stats) == H.HFSEM_ERR_INVALID_ARG
    assert np.all(x == 0.0)
    # freeing NULL handles is a no-op
    lib.hfsem_system_free(None)
    lib.hfsem_factor_free(None)


def test_tile_check_rejects_shapes(lib):
    err = C.c_double(-1.0)
    for N, K, reps in ((8, 64, 1), (24, 64, 1), (144, 64, 1), (32, 48, 1), (32, 136, 1),
                       (32, 64, 0), (32, 64, 9)):
        assert lib.hfsem_tc_tile_check(N, K, reps, C.byref(err)) == H.HFSEM_ERR_INVALID_ARG
    assert lib.hfsem_tc_tile_check(32, 64, 1, None) == H.HFSEM_ERR_INVALID_ARG
    assert err.value == -1.0


def test_status_strings_cover_every_code(lib):
    for code in (H.HFSEM_OK, H.HFSEM_ERR_INVALID_ARG, H.HFSEM_ERR_OOM, H.HFSEM_ERR_NOT_CONVERGED,
                 H.HFSEM_ERR_BREAKDOWN, H.HFSEM_ERR_DEVICE, H.HFSEM_ERR_UNSUPPORTED):
        s = lib.hfsem_status_str(code)
        assert isinstance(s, bytes) and len(s) > 0
    assert len(lib.hfsem_status_str(12345)) > 0


def test_last_error_names_the_problem(lib):
    prob, keep = _problem(alpha=2.5)
    arr = (H.hfsem_problem * 1)(prob)
    out = C.c_void_p(None)
    assert lib.hfsem_assemble(1, arr, None, C.byref(out)) == H.HFSEM_ERR_INVALID_ARG
    assert b"alpha" in lib.hfsem_last_error()
    with pytest.raises(H.HfsemError) as ei:
        H.hfsem_assemble([H.make_problem(np.full(4, 0.25), 3, 1.5, 1.5, 0.0)])
    assert ei.value.code == H.HFSEM_ERR_INVALID_ARG and "theta" in str(ei.value)


def test_timing_read_rejects_null_tag(lib):
    ms = C.c_double(-1.0)
    assert lib.hfsem_timing_read(None, C.byref(ms), None, None) == H.HFSEM_ERR_INVALID_ARG
    assert ms.value == -1.0
    assert lib.hfsem_timing_read(b"no-such-kernel", C.byref(ms), None, None) == H.HFSEM_OK
    assert ms.value == 0.0


@pytest.mark.parametrize("bad", [dict(slots=0), dict(slots=65), dict(budget_bytes=-1),
                                 dict(cache_factors=-1), dict(tol=0.0), dict(max_iter=0),
                                 dict(R=0), dict(R=33), dict(build_only=1)])
def test_server_create_rejects_bad_options(lib, bad):
    ho = H.hopts(R=bad.get("R", 8), build_only=bad.get("build_only", 0))
    o = H.hfsem_server_opts(bad.get("slots", 4), bad.get("budget_bytes", 0),
                            bad.get("cache_factors", 8), ho, bad.get("tol", 1e-12),
                            bad.get("max_iter", 50))
    out = C.c_void_p()
    assert lib.hfsem_server_create(C.byref(o), C.byref(out)) == H.HFSEM_ERR_INVALID_ARG
    assert out.value is None


def test_server_null_handles(lib):
    out = C.c_void_p()
    assert lib.hfsem_server_create(None, C.byref(out)) == H.HFSEM_ERR_INVALID_ARG
    rid = C.c_int64(-7)
    assert lib.hfsem_server_submit(None, None, C.byref(rid)) == H.HFSEM_ERR_INVALID_ARG
    assert rid.value == -7
    n = C.c_int32(-1)
    d = (H.hfsem_done * 4)()
    assert lib.hfsem_server_poll(None, 4, d, C.byref(n)) == H.HFSEM_ERR_INVALID_ARG
    assert lib.hfsem_server_drain(None) == H.HFSEM_ERR_INVALID_ARG
    c = H.hfsem_server_counters()
    assert lib.hfsem_server_counters_read(None, C.byref(c)) == H.HFSEM_ERR_INVALID_ARG
    lib.hfsem_server_free(None)
