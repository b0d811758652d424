"""Python binding of the GB300 non-Hermitian FEAST library (include/feast_gb300.h).

Argument marshalling only: every step of the method runs in libfeast_gb300.so.
Arrays may be numpy complex128 arrays (host) or torch complex128 CUDA tensors
(device); matrices are passed column-major, as the C ABI expects.  Results come
back as numpy arrays unless ``out_device=True`` is given, in which case they are
torch CUDA tensors.

The functions carry the C names: feast_create, feast_factor, feast_get_factor,
feast_solve_shift, feast_filter, feast_rayleigh_ritz, feast_solve,
feast_get_quadrature, feast_destroy.  The library must be built first
(``paper_1404_2891_gb300.build.build()``); importing this module loads it and
raises if it is missing.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfeast_gb300.so")

FEAST_OK = 0
FEAST_ERR_ARG = 1
FEAST_ERR_ALLOC = 2
FEAST_ERR_SINGULAR_SHIFT = 3
FEAST_ERR_REFINE_NOCONV = 4
FEAST_ERR_M0_TOO_SMALL = 5
FEAST_ERR_NOCONV = 6
FEAST_ERR_NONFINITE = 7
FEAST_ERR_DEVICE_TIMEOUT = 8
FEAST_ERR_CUDA = 9
FEAST_ERR_STATE = 10
FEAST_ERR_TOO_LARGE = 11

RULES = {"trap_mid": 0, "trap_end": 1, "gauss": 2, "custom": 3}
ALGOS = {"R": 0, "BI": 1}
PRECISIONS = {"fp64": 0, "mixed": 1}


class feast_z(ctypes.Structure):
    _fields_ = [("re", ctypes.c_double), ("im", ctypes.c_double)]


class feast_contour(ctypes.Structure):
    _fields_ = [("center", feast_z), ("R", ctypes.c_double), ("aspect", ctypes.c_double),
                ("rule", ctypes.c_int), ("N_e", ctypes.c_int),
                ("nodes", ctypes.POINTER(feast_z)), ("weights", ctypes.POINTER(feast_z)),
                ("q_custom", ctypes.c_int)]


class feast_options(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int), ("precision", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_iter", ctypes.c_int), ("cand_tol", ctypes.c_double), ("panel", ctypes.c_int),
                ("timing", ctypes.c_int), ("symmetric", ctypes.c_int), ("max_refine", ctypes.c_int),
                ("refine_tol", ctypes.c_double), ("shift_begin", ctypes.c_int), ("shift_end", ctypes.c_int),
                ("real_pencil", ctypes.c_int), ("tune_cache", ctypes.c_char_p), ("lu_outer", ctypes.c_int),
                ("panel_cluster", ctypes.c_int), ("deep_solves", ctypes.c_int), ("batch_tc_min", ctypes.c_int),
                ("batch_direct", ctypes.c_int)]


class feast_segment(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("a", feast_z), ("b", feast_z), ("r", ctypes.c_double),
                ("t0", ctypes.c_double), ("t1", ctypes.c_double)]


class feast_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("m_found", ctypes.c_int), ("max_res", ctypes.c_double),
                ("normA", ctypes.c_double), ("t_factor_ms", ctypes.c_double),
                ("t_filter_ms", ctypes.c_double), ("t_rr_ms", ctypes.c_double),
                ("t_total_ms", ctypes.c_double), ("t_update_ms", ctypes.c_double),
                ("update_launches", ctypes.c_int), ("res_hist_len", ctypes.c_int),
                ("res_hist", ctypes.c_double * 64), ("count_hist", ctypes.c_int * 64),
                ("q", ctypes.c_int), ("shift_info", ctypes.c_int * 256), ("refine_sweeps", ctypes.c_int),
                ("refactored", ctypes.c_int), ("lu_outer", ctypes.c_int), ("t_deep_ms", ctypes.c_double),
                ("deep_launches", ctypes.c_int), ("deep_flops", ctypes.c_double), ("deep_bytes", ctypes.c_double),
                ("update_flops", ctypes.c_double), ("update_bytes", ctypes.c_double), ("tuned", ctypes.c_int),
                ("t_rr_phase_ms", ctypes.c_double * 8)]


class FeastError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__(f"{where}: {status_str(status)} ({status})")


_lib = None

# every symbol declared in include/feast_gb300.h
SYMBOLS = ("feast_default_options", "feast_create", "feast_destroy", "feast_status_str",
           "feast_get_quadrature", "feast_factor", "feast_get_factor", "feast_solve_shift",
           "feast_filter", "feast_rayleigh_ritz", "feast_solve", "feast_kernel_launches",
           "feast_get_stats", "feast_norm2_estimate_static", "feast_moments",
           "feast_mlp_param_count", "feast_mlp_create", "feast_mlp_destroy", "feast_mlp_get_params",
           "feast_mlp_predict", "feast_mlp_grad", "feast_mlp_train",
           "feast_batch_create", "feast_batch_destroy", "feast_batch_factor", "feast_batch_filter",
           "feast_batch_solve", "feast_batch_get_factor", "feast_batch_info", "feast_batch_tc_info", "feast_batch_plan",
           "feast_emulated_zgemm", "feast_orthonormalize", "feast_set_wait_limit", "feast_contour_nodes",
           "feast_piecewise_nodes", "feast_eta_indicator", "feast_filter_combine",
           "feast_candidates")


class feast_batch_stats(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("tasks_factor", ctypes.c_int),
                ("grid", ctypes.c_int), ("graph", ctypes.c_int), ("plan_makespan_us", ctypes.c_double),
                ("t_factor_ms", ctypes.c_double), ("t_iter_ms", ctypes.c_double * 64), ("tuned", ctypes.c_int)]


def load(path=LIB_PATH):
    """Load the shared library (raises OSError when it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError(f"{path} not found: build it with paper_1404_2891_gb300.build.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.feast_default_options.argtypes = [ctypes.POINTER(feast_options)]
    lib.feast_default_options.restype = None
    lib.feast_create.argtypes = [ctypes.POINTER(P), ctypes.c_int64, P, ctypes.c_int64, P, ctypes.c_int64,
                                 ctypes.POINTER(feast_contour), ctypes.c_int, ctypes.POINTER(feast_options), P]
    lib.feast_create.restype = ctypes.c_int
    lib.feast_destroy.argtypes = [P]
    lib.feast_destroy.restype = None
    lib.feast_status_str.argtypes = [ctypes.c_int]
    lib.feast_status_str.restype = ctypes.c_char_p
    lib.feast_get_quadrature.argtypes = [P, ctypes.POINTER(ctypes.c_int), P, P]
    lib.feast_get_quadrature.restype = ctypes.c_int
    lib.feast_factor.argtypes = [P]
    lib.feast_factor.restype = ctypes.c_int
    lib.feast_get_factor.argtypes = [P, ctypes.c_int, P, P]
    lib.feast_get_factor.restype = ctypes.c_int
    lib.feast_solve_shift.argtypes = [P, ctypes.c_int, ctypes.c_int, P, P, ctypes.c_int]
    lib.feast_solve_shift.restype = ctypes.c_int
    lib.feast_filter.argtypes = [P, P, P, P, P, P]
    lib.feast_filter.restype = ctypes.c_int
    lib.feast_rayleigh_ritz.argtypes = [P, P, P, P, P, P, P, ctypes.POINTER(ctypes.c_int)]
    lib.feast_rayleigh_ritz.restype = ctypes.c_int
    lib.feast_solve.argtypes = [P, P, P, P, P, P, P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(feast_stats)]
    lib.feast_solve.restype = ctypes.c_int
    lib.feast_kernel_launches.argtypes = []
    lib.feast_kernel_launches.restype = ctypes.c_uint64
    lib.feast_get_stats.argtypes = [P, ctypes.POINTER(feast_stats)]
    lib.feast_get_stats.restype = ctypes.c_int
    lib.feast_norm2_estimate_static.argtypes = [P, ctypes.c_int64, ctypes.c_int64, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_double), P]
    lib.feast_norm2_estimate_static.restype = ctypes.c_int
    lib.feast_moments.argtypes = [P, P, ctypes.c_int, ctypes.c_int, P]
    lib.feast_moments.restype = ctypes.c_int
    I = ctypes.c_int
    lib.feast_mlp_param_count.argtypes = [I, I]
    lib.feast_mlp_param_count.restype = ctypes.c_size_t
    lib.feast_mlp_create.argtypes = [ctypes.POINTER(P), I, I, I, P, P, P, P]
    lib.feast_mlp_create.restype = I
    lib.feast_mlp_destroy.argtypes = [P]
    lib.feast_mlp_destroy.restype = None
    lib.feast_mlp_get_params.argtypes = [P, P]
    lib.feast_mlp_get_params.restype = I
    lib.feast_mlp_predict.argtypes = [P, P, I, P]
    lib.feast_mlp_predict.restype = I
    lib.feast_mlp_grad.argtypes = [P, P, P, I, P, P]
    lib.feast_mlp_grad.restype = I
    lib.feast_mlp_train.argtypes = [P, P, P, I, P, I, I, ctypes.c_float, P]
    lib.feast_mlp_train.restype = I
    lib.feast_batch_create.argtypes = [ctypes.POINTER(P), I, P, P, P, P, P, ctypes.POINTER(feast_options), P]
    lib.feast_batch_create.restype = I
    lib.feast_batch_destroy.argtypes = [P]
    lib.feast_batch_destroy.restype = None
    lib.feast_batch_factor.argtypes = [P]
    lib.feast_batch_factor.restype = I
    lib.feast_batch_filter.argtypes = [P, P, P]
    lib.feast_batch_filter.restype = I
    lib.feast_batch_solve.argtypes = [P, P, P, P, P, P, ctypes.POINTER(feast_batch_stats)]
    lib.feast_batch_solve.restype = I
    lib.feast_batch_get_factor.argtypes = [P, I, I, P, P]
    lib.feast_batch_get_factor.restype = I
    lib.feast_batch_info.argtypes = [P, P, P, P, P, P, P]
    lib.feast_batch_info.restype = I
    lib.feast_batch_tc_info.argtypes = [P, P, P, P]
    lib.feast_batch_tc_info.restype = I
    lib.feast_batch_plan.argtypes = [I, P, P, I, I, I, P, I, P, P]
    lib.feast_batch_plan.restype = I
    I64 = ctypes.c_int64
    lib.feast_emulated_zgemm.argtypes = [I64, I64, P, I64, I, P, I64, P, I64, P]
    lib.feast_emulated_zgemm.restype = I
    lib.feast_orthonormalize.argtypes = [I64, I64, P, I64, P]
    lib.feast_orthonormalize.restype = I
    lib.feast_set_wait_limit.argtypes = [ctypes.c_double]
    lib.feast_set_wait_limit.restype = None
    lib.feast_contour_nodes.argtypes = [ctypes.POINTER(feast_contour), ctypes.POINTER(ctypes.c_int), P, P]
    lib.feast_contour_nodes.restype = I
    lib.feast_piecewise_nodes.argtypes = [ctypes.POINTER(feast_segment), I, I, I, ctypes.POINTER(ctypes.c_int), P, P]
    lib.feast_piecewise_nodes.restype = I
    lib.feast_eta_indicator.argtypes = [ctypes.POINTER(feast_contour), P, I, I, P]
    lib.feast_eta_indicator.restype = I
    lib.feast_filter_combine.argtypes = [P, I, P, P, P, P, P, P, P]
    lib.feast_filter_combine.restype = I
    lib.feast_candidates.argtypes = [P, ctypes.POINTER(ctypes.c_int), P, ctypes.POINTER(ctypes.c_double)]
    lib.feast_candidates.restype = I
    _lib = lib
    return lib


def feast_kernel_launches():
    """Kernels launched by the library in this process so far."""
    return int(load().feast_kernel_launches())


def status_str(s):
    return load().feast_status_str(int(s)).decode()


def _check(status, where, allow=()):
    if status != FEAST_OK and status not in allow:
        raise FeastError(status, where)
    return status


# ---------------------------------------------------------------- marshalling
def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _colmajor(x):
    """(pointer, keepalive) for a 1-D or 2-D complex128 array in column-major order."""
    if x is None:
        return None, None
    if _is_torch(x):
        import torch
        t = x
        if t.dtype != torch.complex128:
            raise TypeError("torch inputs must be complex128")
        if t.dim() == 2:
            t = t.mT.contiguous()  # row-major storage of A^T = column-major storage of A
        else:
            t = t.contiguous()
        return t.data_ptr(), t
    a = np.asarray(x, dtype=np.complex128)
    a = np.asfortranarray(a) if a.ndim == 2 else np.ascontiguousarray(a)
    return a.ctypes.data, a


def _out(shape, device, dtype=np.complex128):
    if device:
        import torch
        tdt = torch.complex128 if dtype == np.complex128 else (torch.float64 if dtype == np.float64 else torch.int32)
        t = torch.empty(tuple(reversed(shape)), dtype=tdt, device="cuda")  # column-major view later
        return t.data_ptr(), t
    a = np.zeros(shape, dtype=dtype, order="F")
    return a.ctypes.data, a


def _finish(buf, device):
    if device:
        return buf.mT if buf.dim() == 2 else buf
    return buf


class Handle:
    """Owns a feast_handle*; freed by feast_destroy or garbage collection."""

    def __init__(self, ptr, n, m0, q, algo):
        self.ptr, self.n, self.m0, self.q, self.algo = ptr, n, m0, q, algo

    def __del__(self):
        try:
            feast_destroy(self)
        except Exception:
            pass


def make_contour(center=0.0, R=1.0, aspect=1.0, rule="trap_mid", N_e=8, nodes=None, weights=None):
    c = feast_contour()
    c.center = feast_z(complex(center).real, complex(center).imag)
    c.R, c.aspect = float(R), float(aspect)
    c.rule = RULES[rule]
    c.N_e = int(N_e)
    c._keep = []
    if rule == "custom":
        nz = (feast_z * len(nodes))(*[feast_z(complex(v).real, complex(v).imag) for v in nodes])
        wz = (feast_z * len(weights))(*[feast_z(complex(v).real, complex(v).imag) for v in weights])
        c.nodes = ctypes.cast(nz, ctypes.POINTER(feast_z))
        c.weights = ctypes.cast(wz, ctypes.POINTER(feast_z))
        c.q_custom = len(nodes)
        c._keep = [nz, wz]
    return c


def make_options(algo="BI", precision="mixed", tol=1e-10, max_iter=20, cand_tol=1e-4, panel=0, timing=False,
                 symmetric=False, max_refine=0, refine_tol=1e-12, shifts=None, real_pencil=False, tune_cache=None,
                 lu_outer=0, panel_cluster=0, deep_solves=0, batch_tc_min=0, batch_direct=False):
    """shifts: (begin, end) range of the contour's nodes this handle owns (None = all)."""
    o = feast_options()
    load().feast_default_options(ctypes.byref(o))
    o.algo = ALGOS[algo]
    o.precision = PRECISIONS[precision]
    o.tol, o.max_iter, o.cand_tol, o.panel, o.timing = float(tol), int(max_iter), float(cand_tol), int(panel), int(timing)
    o.symmetric = int(symmetric)
    o.max_refine, o.refine_tol = int(max_refine), float(refine_tol)
    if shifts is not None:
        o.shift_begin, o.shift_end = int(shifts[0]), int(shifts[1])
    o.real_pencil = int(real_pencil)
    o.tune_cache = None if tune_cache is None else str(tune_cache).encode()
    o.lu_outer = int(lu_outer)
    o.panel_cluster = int(panel_cluster)
    o.deep_solves = int(deep_solves)
    o.batch_tc_min = int(batch_tc_min)
    o.batch_direct = int(batch_direct)
    return o


# ---------------------------------------------------------------- entry points
def feast_create(A, B, contour, m0, options, stream=None):
    """feast_create: A, B (None = identity) n x n complex128; contour from make_contour;
    options from make_options; stream: torch.cuda.Stream or raw cudaStream_t (int) or None."""
    lib = load()
    n = A.shape[0]
    pa, ka = _colmajor(A)
    pb, kb = _colmajor(B)
    h = ctypes.c_void_p()
    sp = None
    if stream is not None:
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    s = lib.feast_create(ctypes.byref(h), n, pa, n, pb, n, ctypes.byref(contour), int(m0),
                         ctypes.byref(options), sp)
    _check(s, "feast_create")
    q = ctypes.c_int()
    lib.feast_get_quadrature(h, ctypes.byref(q), None, None)
    return Handle(h, n, int(m0), q.value, options.algo)


def feast_destroy(h):
    if h is not None and h.ptr:
        load().feast_destroy(h.ptr)
        h.ptr = None


def feast_get_quadrature(h):
    lib = load()
    q = h.q
    nodes = (feast_z * q)()
    weights = (feast_z * q)()
    _check(lib.feast_get_quadrature(h.ptr, None, nodes, weights), "feast_get_quadrature")
    z = np.array([complex(v.re, v.im) for v in nodes])
    w = np.array([complex(v.re, v.im) for v in weights])
    return z, w


def feast_get_stats(h):
    st = feast_stats()
    _check(load().feast_get_stats(h.ptr, ctypes.byref(st)), "feast_get_stats")
    return dict(normA=st.normA, t_factor_ms=st.t_factor_ms, t_update_ms=st.t_update_ms,
                update_launches=st.update_launches, t_filter_ms=st.t_filter_ms, t_rr_ms=st.t_rr_ms,
                q=st.q, shift_info=list(st.shift_info[:st.q]), refine_sweeps=st.refine_sweeps,
                refactored=st.refactored, lu_outer=st.lu_outer, t_deep_ms=st.t_deep_ms,
                t_rr_phase_ms=list(st.t_rr_phase_ms),
                deep_launches=st.deep_launches, deep_flops=st.deep_flops, deep_bytes=st.deep_bytes,
                update_flops=st.update_flops, update_bytes=st.update_bytes, tuned=st.tuned)


def feast_set_wait_limit(seconds):
    """Time limit of the library's cross-CTA waits (<= 0: built-in limits)."""
    load().feast_set_wait_limit(float(seconds))


def feast_contour_nodes(contour):
    """(nodes, weights) of a contour from make_contour, computed by the library on the host."""
    lib = load()
    q = ctypes.c_int()
    _check(lib.feast_contour_nodes(ctypes.byref(contour), ctypes.byref(q), None, None), "feast_contour_nodes")
    nz, wz = (feast_z * q.value)(), (feast_z * q.value)()
    _check(lib.feast_contour_nodes(ctypes.byref(contour), ctypes.byref(q), nz, wz), "feast_contour_nodes")
    return (np.array([complex(v.re, v.im) for v in nz]), np.array([complex(v.re, v.im) for v in wz]))


def feast_norm2_estimate_static(A, iters=50, stream=None):
    """||A||_2 by the power iteration of feast_create, without any device
    allocation: for callers that may not call cudaMalloc (the scratch lives in
    a fixed 520.5 KiB device array of the library; n <= 16384).  A must be a
    complex128 CUDA tensor whose storage is column-major (e.g. ``T.mT`` of a
    contiguous tensor T holding A^T); no copy of A is made."""
    if not _is_torch(A) or not A.is_cuda:
        raise TypeError("feast_norm2_estimate_static needs a CUDA tensor (device memory)")
    import torch
    if A.dtype != torch.complex128 or A.dim() != 2:
        raise TypeError("A must be a 2-D complex128 CUDA tensor")
    if A.shape[0] != A.shape[1]:
        raise TypeError(f"A must be square, got {tuple(A.shape)}")
    n = A.shape[0]
    # column-major storage: unit row stride, column stride lda >= n
    if n > 1 and (A.stride(0) != 1 or A.stride(1) < n):
        raise TypeError("A must have column-major storage (unit row stride, column stride >= n)")
    lda = max(int(A.stride(1)), n)
    out = ctypes.c_double()
    sp = None
    if stream is not None:
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(load().feast_norm2_estimate_static(A.data_ptr(), n, lda, int(iters), ctypes.byref(out), sp),
           "feast_norm2_estimate_static")
    return out.value


def feast_piecewise_nodes(segments, K, rule="trap_end"):
    """Nodes and weights of a glued contour (Sec. 5.4).  segments: list of
    ("line", z0, z1) or ("arc", c, r, th0, th1); rule "trap_end" or "gauss"."""
    lib = load()
    segs = (feast_segment * len(segments))()
    for i, sg in enumerate(segments):
        g = segs[i]
        if sg[0] == "line":
            g.kind = 0
            g.a = feast_z(complex(sg[1]).real, complex(sg[1]).imag)
            g.b = feast_z(complex(sg[2]).real, complex(sg[2]).imag)
        else:
            g.kind = 1
            g.a = feast_z(complex(sg[1]).real, complex(sg[1]).imag)
            g.r, g.t0, g.t1 = float(sg[2]), float(sg[3]), float(sg[4])
    q = ctypes.c_int()
    _check(lib.feast_piecewise_nodes(segs, len(segments), int(K), RULES[rule], ctypes.byref(q), None, None),
           "feast_piecewise_nodes")
    nz, wz = (feast_z * q.value)(), (feast_z * q.value)()
    _check(lib.feast_piecewise_nodes(segs, len(segments), int(K), RULES[rule], ctypes.byref(q), nz, wz),
           "feast_piecewise_nodes")
    return (np.array([complex(v.re, v.im) for v in nz]), np.array([complex(v.re, v.im) for v in wz]))


def feast_eta_indicator(contour, r, ntheta=720):
    """eta(r) of Sec. 3 for a contour from make_contour (host computation in the library)."""
    rr = np.ascontiguousarray(r, dtype=np.float64)
    eta = np.zeros_like(rr)
    _check(load().feast_eta_indicator(ctypes.byref(contour), rr.ctypes.data, len(rr), int(ntheta), eta.ctypes.data),
           "feast_eta_indicator")
    return eta


def feast_factor(h, allow_singular=False):
    allow = (FEAST_ERR_SINGULAR_SHIFT,) if allow_singular else ()
    return _check(load().feast_factor(h.ptr), "feast_factor", allow)


def feast_get_factor(h, k):
    LU = np.zeros((h.n, h.n), dtype=np.complex128, order="F")
    piv = np.zeros(h.n, dtype=np.int32)
    _check(load().feast_get_factor(h.ptr, int(k), LU.ctypes.data, piv.ctypes.data), "feast_get_factor")
    return LU, piv


def feast_solve_shift(h, k, side, R, out_device=False):
    pr, kr = _colmajor(R)
    nrhs = R.shape[1] if R.ndim == 2 else 1
    px, X = _out((h.n, nrhs), out_device)
    _check(load().feast_solve_shift(h.ptr, int(k), int(side), pr, px, nrhs), "feast_solve_shift")
    return _finish(X, out_device)


def feast_moments(h, V, kmax):
    """mu_0 .. mu_kmax of the filter from the probe block V (n x S)."""
    pv, kv = _colmajor(V)
    S = V.shape[1] if V.ndim == 2 else 1
    mu = np.zeros(kmax + 1, dtype=np.complex128)
    _check(load().feast_moments(h.ptr, pv, S, int(kmax), mu.ctypes.data), "feast_moments")
    return mu


def feast_filter(h, Y, Yhat=None, theta=None, out_device=False):
    py, ky = _colmajor(Y)
    pyh, kyh = _colmajor(Yhat)
    pt, kt = _colmajor(theta)
    pq, Q = _out((h.n, h.m0), out_device)
    pqh, Qh = (_out((h.n, h.m0), out_device) if Yhat is not None else (None, None))
    _check(load().feast_filter(h.ptr, py, pyh, pt, pq, pqh), "feast_filter")
    return _finish(Q, out_device), (_finish(Qh, out_device) if Yhat is not None else None)


def feast_filter_combine(h, parts, parts_hat=None, Y=None, Yhat=None, theta=None, out_device=False):
    """Sum the partial filters of a shift partition along the fixed tree (see
    include/feast_gb300.h); parts (and parts_hat) list the n x m0 blocks in the
    order of their shift ranges."""
    keep = [_colmajor(p) for p in parts]
    keeph = [_colmajor(p) for p in parts_hat] if parts_hat is not None else None
    py, ky = _colmajor(Y)
    pyh, kyh = _colmajor(Yhat)
    pt, kt = _colmajor(theta)
    pq, Q = _out((h.n, h.m0), out_device)
    pqh, Qh = (_out((h.n, h.m0), out_device) if parts_hat is not None else (None, None))
    _check(load().feast_filter_combine(h.ptr, len(parts), _ptr_array([k[0] for k in keep]),
                                       _ptr_array([k[0] for k in keeph]) if keeph is not None else None,
                                       py, pyh, pt, pq, pqh), "feast_filter_combine")
    return _finish(Q, out_device), (_finish(Qh, out_device) if parts_hat is not None else None)


def feast_rayleigh_ritz(h, Q, Qhat=None, out_device=False):
    pq, kq = _colmajor(Q)
    pqh, kqh = _colmajor(Qhat)
    lam = np.zeros(h.m0, dtype=np.complex128)
    res = np.zeros(h.m0, dtype=np.float64)
    px, X = _out((h.n, h.m0), out_device)
    pxl, Xl = (_out((h.n, h.m0), out_device) if Qhat is not None else (None, None))
    mi = ctypes.c_int()
    _check(load().feast_rayleigh_ritz(h.ptr, pq, pqh, lam.ctypes.data, px, pxl, res.ctypes.data,
                                      ctypes.byref(mi)), "feast_rayleigh_ritz")
    return dict(lam=lam, X=_finish(X, out_device), Xl=_finish(Xl, out_device) if Qhat is not None else None,
                res=res, m_inside=mi.value)


def feast_candidates(h):
    """(indices sorted by (Re, Im), max normalised residual) of the last Rayleigh-Ritz step's candidates."""
    c = ctypes.c_int()
    idx = np.zeros(h.m0, dtype=np.int32)
    mr = ctypes.c_double()
    _check(load().feast_candidates(h.ptr, ctypes.byref(c), idx.ctypes.data, ctypes.byref(mr)), "feast_candidates")
    return idx[:c.value].astype(np.int64), mr.value


def feast_solve(h, Y0, Vrand=None, out_device=False, allow_noconv=True):
    py, ky = _colmajor(Y0)
    pv, kv = _colmajor(Vrand)
    lam = np.zeros(h.m0, dtype=np.complex128)
    res = np.zeros(h.m0, dtype=np.float64)
    px, X = _out((h.n, h.m0), out_device)
    pxl, Xl = (_out((h.n, h.m0), out_device) if h.algo == ALGOS["BI"] else (None, None))
    mf = ctypes.c_int()
    st = feast_stats()
    s = load().feast_solve(h.ptr, py, pv, lam.ctypes.data, px, pxl, res.ctypes.data, ctypes.byref(mf),
                           ctypes.byref(st))
    _check(s, "feast_solve", (FEAST_ERR_NOCONV, FEAST_ERR_M0_TOO_SMALL) if allow_noconv else ())
    k = mf.value
    Xf = _finish(X, out_device)
    out = dict(status=s, converged=(s == FEAST_OK), m_found=k, lam=lam[:k], res=res[:k],
               shift_info=list(st.shift_info[:st.q]), refine_sweeps=st.refine_sweeps, refactored=st.refactored,
               X=Xf[:, :k], iters=st.iters, max_res=st.max_res, normA=st.normA,
               t_factor_ms=st.t_factor_ms, t_filter_ms=st.t_filter_ms, t_rr_ms=st.t_rr_ms,
               t_total_ms=st.t_total_ms,
               res_hist=list(st.res_hist[:st.res_hist_len]), count_hist=list(st.count_hist[:st.res_hist_len]))
    if Xl is not None:
        out["Xl"] = _finish(Xl, out_device)[:, :k]
    return out


# ---------------------------------------------------------------- batched path
class Batch:
    """Owns a feast_batch* (many standard pencils, R-FEAST, mixed precision)."""

    def __init__(self, ptr, n, m0, keep):
        self.ptr, self.n, self.m0, self._keep = ptr, list(n), list(m0), keep

    def __del__(self):
        try:
            feast_batch_destroy(self)
        except Exception:
            pass


def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * len(ptrs))(*[ctypes.c_void_p(p) if p else None for p in ptrs])
    return arr


def feast_batch_create(As, contours, m0, options, stream=None):
    """As: list of n_p x n_p complex128 matrices (numpy or torch CUDA); contours:
    list of make_contour results; m0: list of subspace sizes; options from
    make_options(algo="R", precision="mixed", ...)."""
    lib = load()
    count = len(As)
    keep = [_colmajor(A) for A in As]
    n = np.array([A.shape[0] for A in As], dtype=np.int64)
    lda = n.copy()
    ptrs = _ptr_array([k[0] for k in keep])
    cons = (feast_contour * count)(*contours)
    m = np.array(m0, dtype=np.int32)
    b = ctypes.c_void_p()
    sp = None
    if stream is not None:
        sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(lib.feast_batch_create(ctypes.byref(b), count, n.ctypes.data, ptrs, lda.ctypes.data, cons, m.ctypes.data,
                                  ctypes.byref(options), sp), "feast_batch_create")
    return Batch(b, n.tolist(), m.tolist(), (keep, contours))


def feast_batch_destroy(b):
    if b is not None and b.ptr:
        load().feast_batch_destroy(b.ptr)
        b.ptr = None


def feast_batch_factor(b, allow_singular=False):
    allow = (FEAST_ERR_SINGULAR_SHIFT,) if allow_singular else ()
    return _check(load().feast_batch_factor(b.ptr), "feast_batch_factor", allow)


def feast_batch_filter(b, Ys):
    """Plain filter Q_p = sum_k w_k (z_k I - A_p)^{-1} Y_p for every pencil."""
    keep = [_colmajor(Y) for Y in Ys]
    outs = [np.zeros((n, m), dtype=np.complex128, order="F") for n, m in zip(b.n, b.m0)]
    _check(load().feast_batch_filter(b.ptr, _ptr_array([k[0] for k in keep]),
                                     _ptr_array([o.ctypes.data for o in outs])), "feast_batch_filter")
    return outs


def feast_batch_solve(b, Y0s, allow_noconv=True):
    keep = [_colmajor(Y) for Y in Y0s]
    lams = [np.zeros(m, dtype=np.complex128) for m in b.m0]
    ress = [np.zeros(m, dtype=np.float64) for m in b.m0]
    Xs = [np.zeros((n, m), dtype=np.complex128, order="F") for n, m in zip(b.n, b.m0)]
    mf = np.zeros(len(b.n), dtype=np.int32)
    st = feast_batch_stats()
    s = load().feast_batch_solve(b.ptr, _ptr_array([k[0] for k in keep]), _ptr_array([l.ctypes.data for l in lams]),
                                 _ptr_array([x.ctypes.data for x in Xs]), _ptr_array([r.ctypes.data for r in ress]),
                                 mf.ctypes.data, ctypes.byref(st))
    _check(s, "feast_batch_solve", (FEAST_ERR_NOCONV,) if allow_noconv else ())
    out = []
    for p in range(len(b.n)):
        k = int(mf[p])
        out.append(dict(m_found=k, lam=lams[p][:k], res=ress[p][:k], X=Xs[p][:, :k]))
    stats = dict(status=s, converged=st.converged, iters=st.iters, tasks_factor=st.tasks_factor, grid=st.grid,
                 graph=st.graph, plan_makespan_us=st.plan_makespan_us, t_factor_ms=st.t_factor_ms,
                 t_iter_ms=list(st.t_iter_ms[:st.iters]), tuned=st.tuned)
    return out, stats


def feast_batch_get_factor(b, p, k):
    n = b.n[p]
    LU = np.zeros((n, n), dtype=np.complex128, order="F")
    perm = np.zeros(n, dtype=np.int32)
    _check(load().feast_batch_get_factor(b.ptr, int(p), int(k), LU.ctypes.data, perm.ctypes.data),
           "feast_batch_get_factor")
    return LU, perm


def feast_batch_info(b):
    c, nm, g, t = (ctypes.c_int() for _ in range(4))
    mk, fl = ctypes.c_double(), ctypes.c_double()
    _check(load().feast_batch_info(b.ptr, ctypes.byref(c), ctypes.byref(nm), ctypes.byref(g), ctypes.byref(t),
                                   ctypes.byref(mk), ctypes.byref(fl)), "feast_batch_info")
    return dict(count=c.value, nmat=nm.value, grid=g.value, tasks_factor=t.value, plan_makespan_us=mk.value,
                lu_flops=fl.value)


def feast_batch_tc_info(b):
    """The batch's tensor-core classes: tc_min (0 = none), classes, matrices."""
    t, c, m = (ctypes.c_int() for _ in range(3))
    _check(load().feast_batch_tc_info(b.ptr, ctypes.byref(t), ctypes.byref(c), ctypes.byref(m)),
           "feast_batch_tc_info")
    return dict(tc_min=t.value, classes=c.value, matrices=m.value)


def feast_batch_plan(nb, m, with_lu=True, with_solve=True, workers=152):
    """The host scheduler alone: (tasks as an (ntasks, 4) int array, model makespan in us)."""
    lib = load()
    nbv = np.ascontiguousarray(nb, dtype=np.int32)
    mv = np.ascontiguousarray(m, dtype=np.int32)
    nt = ctypes.c_int()
    mk = ctypes.c_double()
    _check(lib.feast_batch_plan(len(nbv), nbv.ctypes.data, mv.ctypes.data, int(with_lu), int(with_solve),
                                int(workers), None, 0, ctypes.byref(nt), ctypes.byref(mk)), "feast_batch_plan")
    out = np.zeros((nt.value, 4), dtype=np.int32)
    _check(lib.feast_batch_plan(len(nbv), nbv.ctypes.data, mv.ctypes.data, int(with_lu), int(with_solve),
                                int(workers), out.ctypes.data, nt.value, ctypes.byref(nt), ctypes.byref(mk)),
           "feast_batch_plan")
    return out, mk.value


def feast_emulated_zgemm(A, X, op="N"):
    """op(A) X (op "N" or "C") by the emulated-FP64 tensor-core product (diagnostic)."""
    pa, ka = _colmajor(A)
    px, kx = _colmajor(X)
    n = A.shape[0]
    m = X.shape[1] if X.ndim == 2 else 1
    C = np.zeros((n, m), dtype=np.complex128, order="F")
    _check(load().feast_emulated_zgemm(n, m, pa, n, {"N": 0, "C": 2}[op], px, n, C.ctypes.data, n, None),
           "feast_emulated_zgemm")
    return C


def feast_orthonormalize(Q):
    """Orthonormal basis of Q's columns by the library's FP64 CGS2 (diagnostic)."""
    Q = np.array(Q, dtype=np.complex128, order="F", copy=True)
    n, m = Q.shape
    _check(load().feast_orthonormalize(n, m, Q.ctypes.data, n, None), "feast_orthonormalize")
    return Q


# ---------------------------------------------------------------- count predictor (m0)
class MLP:
    """Owns a feast_mlp* (d_in -> width -> width -> 1).  Features and labels are
    moved to the GPU as float32 torch tensors before the kernels read them."""

    def __init__(self, d_in, width, max_batch, params, mean, scale, stream=None):
        import torch
        self.d_in, self.width, self.max_batch = d_in, width, max_batch
        self.nparam = int(load().feast_mlp_param_count(d_in, width))
        p = np.ascontiguousarray(params, dtype=np.float32)
        assert p.size == self.nparam
        m = np.ascontiguousarray(mean, dtype=np.float32)
        s = np.ascontiguousarray(scale, dtype=np.float32)
        self.ptr = ctypes.c_void_p()
        sp = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
        _check(load().feast_mlp_create(ctypes.byref(self.ptr), d_in, width, max_batch, p.ctypes.data, m.ctypes.data,
                                       s.ctypes.data, sp), "feast_mlp_create")
        self._torch = torch

    def _dev(self, a, dtype):
        t = self._torch
        if isinstance(a, t.Tensor):
            return a.to(device="cuda", dtype=dtype).contiguous()
        return t.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")

    def params(self):
        out = np.zeros(self.nparam, dtype=np.float32)
        _check(load().feast_mlp_get_params(self.ptr, out.ctypes.data), "feast_mlp_get_params")
        return out

    def predict(self, X):
        Xd = self._dev(X, self._torch.float32)
        B = Xd.shape[0]
        y = np.zeros(B, dtype=np.float32)
        _check(load().feast_mlp_predict(self.ptr, Xd.data_ptr(), B, y.ctypes.data), "feast_mlp_predict")
        return y

    def grad(self, X, y):
        Xd, yd = self._dev(X, self._torch.float32), self._dev(y, self._torch.float32)
        loss = ctypes.c_float()
        g = np.zeros(self.nparam, dtype=np.float32)
        _check(load().feast_mlp_grad(self.ptr, Xd.data_ptr(), yd.data_ptr(), Xd.shape[0], ctypes.byref(loss),
                                     g.ctypes.data), "feast_mlp_grad")
        return loss.value, g

    def train(self, X, y, batches, lr):
        """batches: (steps, B) int32 row indices; returns the last mini-batch loss."""
        Xd, yd = self._dev(X, self._torch.float32), self._dev(y, self._torch.float32)
        bd = self._dev(np.asarray(batches, dtype=np.int32), self._torch.int32)
        steps, B = bd.shape
        loss = ctypes.c_float()
        _check(load().feast_mlp_train(self.ptr, Xd.data_ptr(), yd.data_ptr(), Xd.shape[0], bd.data_ptr(), steps, B,
                                      float(lr), ctypes.byref(loss)), "feast_mlp_train")
        return loss.value

    def __del__(self):
        try:
            if self.ptr:
                load().feast_mlp_destroy(self.ptr)
                self.ptr = None
        except Exception:
            pass
