"""Thin Python binding of the hfsem C ABI (include/hfsem.h).

Argument marshalling only: every step of the solver runs in the CUDA library
libhfsem.so.  The functions keep the C names.  Vectors may be numpy arrays
(host) or CUDA torch tensors (device); the library accepts both kinds of
pointer.  If the shared library has not been built, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
import weakref

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhfsem.so")

HFSEM_OK = 0
HFSEM_ERR_INVALID_ARG = 1
HFSEM_ERR_OOM = 2
HFSEM_ERR_NOT_CONVERGED = 3
HFSEM_ERR_BREAKDOWN = 4
HFSEM_ERR_TIMEOUT = 5
HFSEM_ERR_DEVICE = 6
HFSEM_ERR_UNSUPPORTED = 7

MATVEC_AUTO, MATVEC_DENSE, MATVEC_TOEPLITZ, MATVEC_HMATRIX = 0, 1, 2, 3
PREC_FP64, PREC_MIXED, PREC_MIXED_TC = 0, 1, 2   # PREC_MIXED_TC: dense leaf products of the H-LU on the tensor cores
RHS_LOAD_VECTOR, RHS_FRAC_POWERS, RHS_LEGENDRE_AB = 0, 1, 2
ADM_MAX, ADM_MIN = 0, 1   # admissibility: eq. (admis) as printed, or min(diam) <= lambda dist

# every symbol include/hfsem.h declares
EXPORTED = ["hfsem_assemble", "hfsem_ndof", "hfsem_apply", "hfsem_load_vector",
            "hfsem_hlu_factor", "hfsem_hmatrix_dense", "hfsem_precond_apply",
            "hfsem_solve", "hfsem_factor_free", "hfsem_system_free",
            "hfsem_status_str", "hfsem_timing_enable", "hfsem_timing_reset",
            "hfsem_timing_read", "hfsem_apply_noalloc", "hfsem_tc_tile_check",
            "hfsem_last_error", "hfsem_server_create", "hfsem_server_submit",
            "hfsem_server_poll", "hfsem_server_drain", "hfsem_server_counters_read",
            "hfsem_server_free", "hfsem_alu_peak", "hfsem_hlu_solve", "hfsem_tune",
            "hfsem_tune_load", "hfsem_tune_lookup", "hfsem_tune_clear"]


class HfsemError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: status {code}")
        self.code = code


class hfsem_problem(C.Structure):
    _fields_ = [("n_elem", C.c_int32), ("P", C.c_int32), ("a", C.c_double),
                ("b", C.c_double), ("h", C.POINTER(C.c_double)),
                ("alpha", C.c_double), ("theta", C.c_double), ("rho", C.c_double),
                ("c1", C.c_double), ("c2", C.c_double), ("matvec", C.c_int32)]


class hfsem_hopts(C.Structure):
    _fields_ = [("R", C.c_int32), ("lambda_", C.c_double), ("tol_hlu", C.c_double),
                ("precision", C.c_int32), ("leaf_elems", C.c_int32),
                ("kmax", C.c_int32), ("build_only", C.c_int32), ("admissibility", C.c_int32)]


class hfsem_rhs(C.Structure):
    _fields_ = [("kind", C.c_int32), ("nrhs", C.c_int32), ("n_terms", C.c_int32),
                ("data", C.POINTER(C.c_double))]


class hfsem_stats(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32),
                ("rel_residual", C.c_double), ("rel_true_residual", C.c_double)]


class hfsem_tune_entry(C.Structure):
    _fields_ = [("fp64", C.c_int32), ("kind", C.c_int32), ("P", C.c_int32),
                ("leaf_dofs", C.c_int32), ("n_inst", C.c_int32), ("ms", C.c_double),
                ("ms_default", C.c_double)]


class hfsem_server_opts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("budget_bytes", C.c_int64),
                ("cache_factors", C.c_int32), ("hopts", hfsem_hopts), ("tol", C.c_double),
                ("max_iter", C.c_int32)]


class hfsem_request(C.Structure):
    _fields_ = [("prob", C.POINTER(hfsem_problem)), ("rhs", C.POINTER(hfsem_rhs)),
                ("X", C.c_void_p), ("stats", C.POINTER(hfsem_stats))]


class hfsem_done(C.Structure):
    _fields_ = [("id", C.c_int64), ("status", C.c_int32), ("reused", C.c_int32),
                ("t_submit", C.c_double), ("t_start", C.c_double), ("t_done", C.c_double),
                ("msg", C.c_char * 128)]


class hfsem_server_counters(C.Structure):
    _fields_ = [("resident_bytes", C.c_int64), ("inflight_bytes", C.c_int64),
                ("budget_bytes", C.c_int64), ("peak_bytes", C.c_int64),
                ("running", C.c_int32), ("peak_running", C.c_int32), ("cached", C.c_int32),
                ("queued", C.c_int32), ("builds", C.c_int64), ("reuses", C.c_int64),
                ("evictions", C.c_int64), ("rejected", C.c_int64)]


_lib = None


def load_library():
    """Load libhfsem.so; raise if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"CUDA library missing: {LIB_PATH}; run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    vp = C.c_void_p
    lib.hfsem_assemble.argtypes = [C.c_int32, C.POINTER(hfsem_problem), vp, C.POINTER(vp)]
    lib.hfsem_ndof.argtypes = [vp, C.c_int32, C.POINTER(C.c_int32)]
    lib.hfsem_apply.argtypes = [vp, C.c_int32, vp, vp]
    lib.hfsem_apply_noalloc.argtypes = [vp, C.c_int32, vp, vp]
    lib.hfsem_tc_tile_check.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_double)]
    lib.hfsem_load_vector.argtypes = [vp, C.POINTER(hfsem_rhs), C.c_int32, vp]
    lib.hfsem_hlu_factor.argtypes = [vp, C.POINTER(hfsem_hopts), C.POINTER(vp)]
    lib.hfsem_hmatrix_dense.argtypes = [vp, C.c_int32, vp]
    lib.hfsem_precond_apply.argtypes = [vp, C.c_int32, vp, vp]
    lib.hfsem_solve.argtypes = [vp, vp, C.POINTER(hfsem_rhs), C.c_double, C.c_int32, vp,
                                C.POINTER(hfsem_stats)]
    lib.hfsem_factor_free.argtypes = [vp]
    lib.hfsem_factor_free.restype = None
    lib.hfsem_system_free.argtypes = [vp]
    lib.hfsem_system_free.restype = None
    lib.hfsem_status_str.argtypes = [C.c_int]
    lib.hfsem_status_str.restype = C.c_char_p
    lib.hfsem_last_error.restype = C.c_char_p
    lib.hfsem_server_create.argtypes = [C.POINTER(hfsem_server_opts), C.POINTER(vp)]
    lib.hfsem_server_submit.argtypes = [vp, C.POINTER(hfsem_request), C.POINTER(C.c_int64)]
    lib.hfsem_server_poll.argtypes = [vp, C.c_int32, C.POINTER(hfsem_done), C.POINTER(C.c_int32)]
    lib.hfsem_server_drain.argtypes = [vp]
    lib.hfsem_server_counters_read.argtypes = [vp, C.POINTER(hfsem_server_counters)]
    lib.hfsem_server_free.argtypes = [vp]
    lib.hfsem_server_free.restype = None
    lib.hfsem_hlu_solve.argtypes = [vp, vp, C.POINTER(hfsem_rhs), vp]
    lib.hfsem_alu_peak.argtypes = [C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                   C.POINTER(C.c_int32)]
    lib.hfsem_tune.argtypes = [vp, C.POINTER(hfsem_hopts), C.POINTER(hfsem_rhs), C.c_double,
                               C.c_int32, C.c_char_p, C.POINTER(hfsem_tune_entry), C.c_int32,
                               C.POINTER(C.c_int32)]
    lib.hfsem_tune_load.argtypes = [C.c_char_p]
    lib.hfsem_tune_lookup.argtypes = [C.c_int32, C.c_int32, C.c_int32, C.POINTER(C.c_int32)]
    lib.hfsem_timing_enable.argtypes = [C.c_int32]
    lib.hfsem_timing_read.argtypes = [C.c_char_p, C.POINTER(C.c_double),
                                      C.POINTER(C.c_int64), C.POINTER(C.c_double)]
    _lib = lib
    return lib


def _check(code: int, what: str, allow=()):
    if code != HFSEM_OK and code not in allow:
        lib = load_library()
        msg = lib.hfsem_last_error().decode()
        raise HfsemError(code, f"{what}: {lib.hfsem_status_str(code).decode()} ({msg})")
    return code


def _ptr(a):
    """(pointer, is_torch) of a contiguous float64 numpy array or tensor."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("need a C-contiguous float64 array")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("need a contiguous float64 tensor")
        return a.data_ptr()
    raise TypeError(type(a))


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return C.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    return C.c_void_p(int(stream))


class System:
    """Handle to an assembled batch of instances (hfsem_system*)."""

    def __init__(self, handle, problems):
        self.h = handle
        self.problems = problems
        self.ndofs = [int(p.n_elem) * int(p.P) - 1 for p in problems]
        self.factors = weakref.WeakSet()   # freed before the system

    @property
    def total_ndof(self):
        return sum(self.ndofs)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            for f in list(getattr(self, "factors", ())):
                f.free()
            _lib.hfsem_system_free(self.h)
            self.h = None


class Factor:
    """Handle to an H-LU factorisation of every instance of a System
    (hfsem_factor*); freed with it or by free()."""

    def __init__(self, handle, system):
        self.h = handle
        self.system = system
        system.factors.add(self)

    def free(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.hfsem_factor_free(self.h)
            self.h = None

    def __del__(self):
        self.free()


def make_problem(h, P, alpha, theta, rho, a=0.0, b=None, c1=0.0, c2=0.0,
                 matvec=MATVEC_AUTO):
    """One instance: element lengths h (N of them, summing to b - a; b defaults
    to a + sum h), degree P, 1 < alpha < 2, 0 <= theta <= 1, rho >= 0,
    boundary values c1 = u(a), c2 = u(b), operator MATVEC_AUTO / _DENSE /
    _TOEPLITZ / _HMATRIX."""
    h = np.ascontiguousarray(h, dtype=np.float64)
    if b is None:
        b = a + float(h.sum())
    return {"h": h, "P": int(P), "alpha": float(alpha), "theta": float(theta),
            "rho": float(rho), "a": float(a), "b": float(b), "c1": float(c1),
            "c2": float(c2), "matvec": int(matvec)}


def hfsem_assemble(problems, stream=None) -> System:
    """Assemble a batch of make_problem() instances on `stream` (a CUDA stream
    handle; default torch's current stream)."""
    lib = load_library()
    arr = (hfsem_problem * len(problems))()
    keep = []
    for i, p in enumerate(problems):
        h = np.ascontiguousarray(p["h"], dtype=np.float64)
        keep.append(h)
        arr[i] = hfsem_problem(len(h), p["P"], p["a"], p["b"],
                               h.ctypes.data_as(C.POINTER(C.c_double)), p["alpha"],
                               p["theta"], p["rho"], p["c1"], p["c2"], p.get("matvec", 0))
    out = C.c_void_p()
    _check(lib.hfsem_assemble(len(problems), arr, _stream_handle(stream), C.byref(out)),
           "hfsem_assemble")
    return System(out, [arr[i] for i in range(len(problems))])


def hfsem_ndof(sys: System, inst: int) -> int:
    """N_d = N P - 1 of instance inst."""
    nd = C.c_int32()
    _check(load_library().hfsem_ndof(sys.h, inst, C.byref(nd)), "hfsem_ndof")
    return nd.value


def _like(x, n):
    if isinstance(x, np.ndarray):
        return np.zeros(n, dtype=np.float64)
    import torch
    return torch.zeros(n, dtype=torch.float64, device=x.device)


def hfsem_apply(sys: System, x, nrhs: int = 1):
    """y = A x for every instance (zero boundary values); x holds nrhs columns
    of N_d per instance, instances concatenated; y is allocated like x (numpy
    array or tensor on x's device)."""
    y = _like(x, sys.total_ndof * nrhs)
    _check(load_library().hfsem_apply(sys.h, nrhs, _ptr(x), _ptr(y)), "hfsem_apply")
    return y


def hfsem_apply_noalloc(sys: System, x, nrhs: int = 1, out=None):
    """y = A x without device allocation; x (and out) must be CUDA tensors."""
    y = _like(x, sys.total_ndof * nrhs) if out is None else out
    _check(load_library().hfsem_apply_noalloc(sys.h, nrhs, _ptr(x), _ptr(y)),
           "hfsem_apply_noalloc")
    return y


def hfsem_tc_tile_check(N: int, K: int, reps: int = 1) -> float:
    """Max entrywise error of the BF16 tensor-core tile C = A B (128 x K times
    K x N) against FP64, relative to sum_k |a_mk b_kn|."""
    out = C.c_double(-1.0)
    _check(load_library().hfsem_tc_tile_check(N, K, reps, C.byref(out)), "hfsem_tc_tile_check")
    return out.value


def _rhs_array(rhs_list):
    """rhs_list: per instance (kind, nrhs, n_terms, data ndarray)."""
    arr = (hfsem_rhs * len(rhs_list))()
    keep = []
    for i, (kind, nrhs, n_terms, data) in enumerate(rhs_list):
        d = np.ascontiguousarray(data, dtype=np.float64).ravel()
        keep.append(d)
        arr[i] = hfsem_rhs(kind, nrhs, n_terms, d.ctypes.data_as(C.POINTER(C.c_double)))
    return arr, keep


def rhs_frac_powers(terms_per_rhs):
    """[(coef, exponent, 'a'|'b'), ...] per rhs -> (kind, nrhs, n_terms, data).
    Right-hand sides with fewer terms are padded with zero terms."""
    nt = max(len(t) for t in terms_per_rhs)
    data = np.zeros((len(terms_per_rhs), nt, 3))
    for r, terms in enumerate(terms_per_rhs):
        for k, (c, mu, side) in enumerate(terms):
            data[r, k] = (c, mu, 0.0 if side == "a" else 1.0)
    return (RHS_FRAC_POWERS, len(terms_per_rhs), nt, data)


def rhs_legendre(coeffs_per_rhs):
    """f = sum_k g_k L_k(xi_[a,b](x)) per rhs, coefficients g_0..g_K ->
    (kind, nrhs, n_terms, data); shorter lists are padded with zeros."""
    K1 = max(len(c) for c in coeffs_per_rhs)
    data = np.zeros((len(coeffs_per_rhs), K1))
    for r, c in enumerate(coeffs_per_rhs):
        data[r, : len(c)] = c
    return (RHS_LEGENDRE_AB, len(coeffs_per_rhs), K1, data)


def rhs_load_vector(G, nrhs=1):
    """A ready load vector: N_d x nrhs column-major in the unknowns' order."""
    G = np.ascontiguousarray(G, dtype=np.float64)
    return (RHS_LOAD_VECTOR, nrhs, 0, G)


def hfsem_load_vector(sys: System, rhs_list, lifted: int = 0, out=None):
    """G = (f, phi_i) for every instance (rhs_list: one rhs_* tuple per
    instance); lifted = 1 subtracts the boundary lifting's contribution."""
    arr, keep = _rhs_array(rhs_list)
    nrhs = rhs_list[0][1]
    G = np.zeros(sys.total_ndof * nrhs) if out is None else out
    _check(load_library().hfsem_load_vector(sys.h, arr, lifted, _ptr(G)), "hfsem_load_vector")
    return G


def hopts(R=8, lam=1.0, tol_hlu=1e-3, precision=PREC_MIXED, leaf_elems=0, kmax=0,
          build_only=0, admissibility=ADM_MAX):
    """H-matrix / H-LU options: Taylor rank R, admissibility lambda, Tol_HLU,
    PREC_FP64 / PREC_MIXED / PREC_MIXED_TC, elements per leaf and rank cap
    (0 = automatic), build_only = 1 to build the H-matrix without factoring,
    ADM_MAX (eq. (admis)) or ADM_MIN."""
    return hfsem_hopts(R, lam, tol_hlu, precision, leaf_elems, kmax, build_only, admissibility)


def hfsem_hlu_factor(sys: System, opts: hfsem_hopts) -> Factor:
    """H-matrix approximation and H-LU factorisation of every instance."""
    out = C.c_void_p()
    _check(load_library().hfsem_hlu_factor(sys.h, C.byref(opts), C.byref(out)),
           "hfsem_hlu_factor")
    return Factor(out, sys)


def hfsem_hmatrix_dense(fac: Factor, inst: int):
    """The H-matrix of instance inst as a dense N_d x N_d array (factors built
    with build_only = 1)."""
    nd = fac.system.ndofs[inst]
    out = np.zeros(nd * nd)
    _check(load_library().hfsem_hmatrix_dense(fac.h, inst, _ptr(out)), "hfsem_hmatrix_dense")
    return out.reshape(nd, nd, order="F")


def hfsem_precond_apply(fac: Factor, r, nrhs: int = 1):
    """y = U^-1 L^-1 r (the two H-triangular solves) for every instance."""
    y = _like(r, fac.system.total_ndof * nrhs)
    _check(load_library().hfsem_precond_apply(fac.h, nrhs, _ptr(r), _ptr(y)),
           "hfsem_precond_apply")
    return y


def hfsem_hlu_solve(sys: System, fac: Factor, rhs_list, X=None):
    """Direct solve of the H-matrix approximation system A~ X = G by the two
    H-triangular solves (no Krylov iteration); X as in hfsem_solve."""
    arr, keep = _rhs_array(rhs_list)
    nrhs = rhs_list[0][1]
    if X is None:
        X = np.zeros(sys.total_ndof * nrhs)
    _check(load_library().hfsem_hlu_solve(sys.h, fac.h, arr, _ptr(X)), "hfsem_hlu_solve")
    return X


def hfsem_solve(sys: System, fac, rhs_list, tol=1e-14, max_iter=200, X=None,
                allow_fail=False):
    """BiCGSTAB from zero on every instance and right-hand side, right-
    preconditioned by fac (None: unpreconditioned), accepted on the true
    residual.  X (numpy array or CUDA tensor, N_d x nrhs per instance,
    concatenated; allocated on the host when None) receives the solution;
    its previous contents are not used.  Returns (X, per-column stats dicts,
    status); raises HfsemError on failure unless allow_fail."""
    arr, keep = _rhs_array(rhs_list)
    nrhs = rhs_list[0][1]
    if X is None:
        X = np.zeros(sys.total_ndof * nrhs)
    stats = (hfsem_stats * (len(sys.ndofs) * nrhs))()
    code = load_library().hfsem_solve(sys.h, fac.h if fac is not None else None, arr,
                                      tol, max_iter, _ptr(X), stats)
    if not allow_fail:
        _check(code, "hfsem_solve")
    st = [dict(iters=s.iters, status=s.status, rel_residual=s.rel_residual,
               rel_true_residual=s.rel_true_residual) for s in stats]
    return X, st, code


def split(sys: System, v, nrhs: int = 1):
    """Split a concatenated vector into per-instance (N_d, nrhs) column-major views."""
    out, off = [], 0
    if hasattr(v, "detach"):   # a torch tensor, possibly on the GPU
        v = v.detach().cpu().numpy()
    v = np.asarray(v)
    for nd in sys.ndofs:
        out.append(v[off: off + nd * nrhs].reshape(nrhs, nd).T)
        off += nd * nrhs
    return out


def hfsem_tune(sys: System, opts: hfsem_hopts, rhs_list, tol=1e-14, max_iter=100, path=None):
    """Leaf-size autotuner: per class of the system's instances, the fastest
    candidate leaf size enters the process-wide table that later
    factorisations with leaf_elems = 0 use.  Returns this call's choices."""
    arr, keep = _rhs_array(rhs_list)
    cap = 256
    out = (hfsem_tune_entry * cap)()
    n = C.c_int32()
    _check(load_library().hfsem_tune(sys.h, C.byref(opts), arr, tol, max_iter,
                                     path.encode() if path else None, out, cap, C.byref(n)),
           "hfsem_tune")
    return [dict(fp64=e.fp64, kind=e.kind, P=e.P, leaf_dofs=e.leaf_dofs, n_inst=e.n_inst,
                 ms=e.ms, ms_default=e.ms_default) for e in out[:min(n.value, cap)]]


def hfsem_tune_load(path: str):
    _check(load_library().hfsem_tune_load(path.encode()), "hfsem_tune_load")


def hfsem_tune_lookup(fp64: int, kind: int, P: int) -> int:
    d = C.c_int32()
    _check(load_library().hfsem_tune_lookup(fp64, kind, P, C.byref(d)), "hfsem_tune_lookup")
    return d.value


def hfsem_tune_clear():
    _check(load_library().hfsem_tune_clear(), "hfsem_tune_clear")


def hfsem_alu_peak(kind: int):
    """(TFLOP/s, best launch ms, SM count) of an FMA-chain microbenchmark on
    the current device; kind 0 = FP64, 1 = FP32."""
    tf, ms, sms = C.c_double(), C.c_double(), C.c_int32()
    _check(load_library().hfsem_alu_peak(kind, C.byref(tf), C.byref(ms), C.byref(sms)),
           "hfsem_alu_peak")
    return tf.value, ms.value, sms.value


def hfsem_timing_enable(on: bool = True):
    """Per-kernel CUDA-event timing inside the library (for the benchmark)."""
    _check(load_library().hfsem_timing_enable(1 if on else 0), "hfsem_timing_enable")


def hfsem_timing_reset():
    _check(load_library().hfsem_timing_reset(), "hfsem_timing_reset")


def hfsem_timing_read(tag: str):
    """(total device ms, launches, algorithmic work) for one kernel tag."""
    ms, n, w = C.c_double(), C.c_int64(), C.c_double()
    _check(load_library().hfsem_timing_read(tag.encode(), C.byref(ms), C.byref(n), C.byref(w)),
           "hfsem_timing_read")
    return ms.value, n.value, w.value


class Server:
    """A serving loop (hfsem_server*): requests, each one instance with its
    right-hand sides, run in `slots` concurrent slots on the current device,
    admitted under a device-memory budget, with resident factorisations
    reused by later requests of the same operator."""

    def __init__(self, slots=8, budget_bytes=0, cache_factors=64, hopts_=None, tol=1e-14,
                 max_iter=100):
        lib = load_library()
        o = hfsem_server_opts(slots, budget_bytes, cache_factors,
                              hopts_ if hopts_ is not None else hopts(), tol, max_iter)
        h = C.c_void_p()
        _check(lib.hfsem_server_create(C.byref(o), C.byref(h)), "hfsem_server_create")
        self.h = h
        self._live = {}      # id -> buffers the library writes on completion

    def submit(self, problem, rhs, X=None):
        """Queue one request: problem from make_problem(), rhs one rhs_* tuple
        (its nrhs columns).  X (numpy array or CUDA tensor, N_d x nrhs) receives
        the solution; allocated on the host when None.  Returns the id."""
        lib = load_library()
        hh = np.ascontiguousarray(problem["h"], dtype=np.float64)
        prob = hfsem_problem(len(hh), problem["P"], problem["a"], problem["b"],
                             hh.ctypes.data_as(C.POINTER(C.c_double)), problem["alpha"],
                             problem["theta"], problem["rho"], problem["c1"], problem["c2"],
                             problem.get("matvec", 0))
        arr, keep = _rhs_array([rhs])
        nrhs = rhs[1]
        nd = len(hh) * problem["P"] - 1
        if X is None:
            X = np.zeros(nd * nrhs)
        elif hasattr(X, "is_cuda") and X.is_cuda:
            # the server writes X from its own streams: work queued on X by
            # the caller's stream (its allocation, a fill) must be done first
            import torch
            torch.cuda.current_stream(X.device).synchronize()
        stats = (hfsem_stats * nrhs)()
        req = hfsem_request(C.pointer(prob), C.cast(arr, C.POINTER(hfsem_rhs)), _ptr(X), stats)
        rid = C.c_int64()
        _check(lib.hfsem_server_submit(self.h, C.byref(req), C.byref(rid)), "hfsem_server_submit")
        self._live[rid.value] = (X, stats)
        return rid.value

    def poll(self, max_n=4096):
        """Completed requests since the last poll: dicts with id, status,
        reused, t_submit / t_start / t_done (seconds), msg, X, stats."""
        lib = load_library()
        out = (hfsem_done * max_n)()
        n = C.c_int32()
        _check(lib.hfsem_server_poll(self.h, max_n, out, C.byref(n)), "hfsem_server_poll")
        res = []
        for d in out[: n.value]:
            X, st = self._live.pop(d.id)
            res.append(dict(id=d.id, status=d.status, reused=d.reused, t_submit=d.t_submit,
                            t_start=d.t_start, t_done=d.t_done, msg=d.msg.decode(), X=X,
                            stats=[dict(iters=s.iters, status=s.status,
                                        rel_residual=s.rel_residual,
                                        rel_true_residual=s.rel_true_residual) for s in st]))
        return res

    def drain(self):
        """Block until every submitted request has completed."""
        _check(load_library().hfsem_server_drain(self.h), "hfsem_server_drain")

    def counters(self):
        c = hfsem_server_counters()
        _check(load_library().hfsem_server_counters_read(self.h, C.byref(c)),
               "hfsem_server_counters_read")
        return {k: getattr(c, k) for k, _ in hfsem_server_counters._fields_}

    def close(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.hfsem_server_free(self.h)
            self.h = None

    def __del__(self):
        self.close()
