"""Python binding of the GB300 matrix-free Karhunen–Loève library (libkl.so).

Argument marshalling only: every function here calls the C ABI of
``include/kl.h`` with the same name, and all computation runs in the
library's CUDA kernels. Device buffers may be passed as torch CUDA tensors
(their ``data_ptr()`` is used) or as raw integer addresses. A block of k
vectors of length n is a contiguous torch tensor of shape (k, n): read as an
n x k matrix it is column-major with leading dimension n, the C layout.

There is no CPU fallback: if ``libkl.so`` is missing the functions raise.
"""
import ctypes
import os

__all__ = [
    "KLError", "kl_params", "kl_solve_info", "kl_kernel_stats", "params",
    "kl_default_params", "kl_create", "kl_destroy", "kl_dims", "kl_apply_A",
    "kl_apply_Zinv", "kl_apply_Aprime", "kl_eigs", "kl_profile_enable",
    "kl_profile_read", "kl_launch_count", "kl_memory", "kl_last_error",
    "kl_status_string", "kl_measure_peaks", "kl_pairwise_noalloc", "kl_estimate_bytes",
    "kl_serve_config", "kl_serve_result", "kl_serve_stats", "kl_serve_open", "kl_serve_submit",
    "kl_serve_poll", "kl_serve_get_stats", "kl_serve_close", "kl_set_graphs", "kl_set_shared_sms", "kl_block_size",
    "kl_autotune", "kl_sample_size", "kl_sample_points", "kl_sample", "kl_bounds_checked", "kl_debug_set", "library_path",
    "EXPORTED_SYMBOLS",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libkl.so")

KL_OK, KL_ERR_ARG, KL_ERR_CUDA, KL_ERR_OOM = 0, -1, -2, -3
KL_ERR_NOCONV, KL_ERR_NUMERIC, KL_ERR_TIMEOUT, KL_ERR_UNSUPPORTED = -4, -5, -6, -7
KL_WARN_COMPLEX = 1
KL_DEBUG_WAIT_LIMIT, KL_DEBUG_FAIL_ALLOC, KL_DEBUG_NAN_START, KL_DEBUG_PAIR_DENSE = 1, 2, 3, 4

GEOMETRIES = {"cube": 0, "annulus": 1, "half_annulus": 2, "projective_cube": 3}
KERNELS = {"gauss": 0, "exp_sep": 1, "exp": 2, "matern32": 3, "const": 4}
METHODS = {"galerkin": 0, "collocation": 1, "galerkin_std": 2}
PRECISIONS = {"fp64": 0, "fp32": 1, "bf16": 2, "tf32": 3}

# Every entry point declared in include/kl.h.
EXPORTED_SYMBOLS = (
    "kl_default_params", "kl_create", "kl_destroy", "kl_dims", "kl_apply_A",
    "kl_apply_Zinv", "kl_apply_Aprime", "kl_eigs", "kl_profile_enable",
    "kl_profile_read", "kl_launch_count", "kl_memory", "kl_last_error",
    "kl_status_string", "kl_measure_peaks", "kl_pairwise_noalloc", "kl_estimate_bytes",
    "kl_serve_open", "kl_serve_submit", "kl_serve_poll", "kl_serve_get_stats", "kl_serve_close",
    "kl_set_graphs", "kl_set_shared_sms", "kl_block_size", "kl_autotune", "kl_sample_size", "kl_sample_points", "kl_sample",
    "kl_bounds_checked", "kl_debug_set",
)


class KLError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{message} (status {status})")
        self.status = status


class kl_params(ctypes.Structure):
    _fields_ = [
        ("dim", ctypes.c_int),
        ("geometry", ctypes.c_int),
        ("geo", ctypes.c_double * 3),
        ("degree", ctypes.c_int),
        ("elems", ctypes.c_int * 3),
        ("kernel", ctypes.c_int),
        ("sigma", ctypes.c_double),
        ("L", ctypes.c_double),
        ("method", ctypes.c_int),
        ("interp_continuity", ctypes.c_int),
        ("precision", ctypes.c_int),
        ("block_k", ctypes.c_int),
        ("refine", ctypes.c_int),
        ("max_restarts", ctypes.c_int),
        ("seed", ctypes.c_ulonglong),
    ]


class kl_solve_info(ctypes.Structure):
    _fields_ = [
        ("restarts", ctypes.c_int),
        ("applies", ctypes.c_int),
        ("vectors_applied", ctypes.c_int),
        ("converged", ctypes.c_int),
        ("max_resid", ctypes.c_double),
        ("max_imag", ctypes.c_double),
        ("seconds", ctypes.c_double),
    ]


class kl_kernel_stats(ctypes.Structure):
    _fields_ = [
        ("name", ctypes.c_char * 32),
        ("launches", ctypes.c_longlong),
        ("ms", ctypes.c_double),
        ("units", ctypes.c_double),
    ]


class kl_serve_config(ctypes.Structure):
    _fields_ = [
        ("hbm_budget_bytes", ctypes.c_int64),
        ("max_slots", ctypes.c_int),
        ("batch_window_us", ctypes.c_int),
    ]


class kl_serve_result(ctypes.Structure):
    _fields_ = [
        ("request_id", ctypes.c_int64),
        ("status", ctypes.c_int),
        ("M", ctypes.c_int),
        ("applies", ctypes.c_int),
        ("restarts", ctypes.c_int),
        ("max_resid", ctypes.c_double),
        ("queue_ms", ctypes.c_double),
        ("solve_ms", ctypes.c_double),
        ("latency_ms", ctypes.c_double),
        ("est_bytes", ctypes.c_int64),
    ]


class kl_serve_stats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_longlong),
        ("completed", ctypes.c_longlong),
        ("batches", ctypes.c_longlong),
        ("batched_products", ctypes.c_longlong),
        ("max_batch", ctypes.c_int),
        ("max_concurrent", ctypes.c_int),
        ("peak_est_bytes", ctypes.c_int64),
        ("budget_bytes", ctypes.c_int64),
    ]


_lib = None


def library_path():
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(_LIB_PATH)
    vp, i64, c_int, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    sig = {
        "kl_default_params": (None, [ctypes.POINTER(kl_params)]),
        "kl_create": (c_int, [ctypes.POINTER(kl_params), vp, ctypes.POINTER(vp)]),
        "kl_destroy": (c_int, [vp]),
        "kl_dims": (c_int, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "kl_apply_A": (c_int, [vp, vp, i64, vp, i64, c_int]),
        "kl_apply_Zinv": (c_int, [vp, vp, i64, vp, i64, c_int]),
        "kl_apply_Aprime": (c_int, [vp, vp, i64, vp, i64, c_int]),
        "kl_eigs": (c_int, [vp, c_int, dbl, vp, vp, i64, c_int, vp, ctypes.POINTER(kl_solve_info)]),
        "kl_profile_enable": (c_int, [vp, c_int]),
        "kl_profile_read": (c_int, [vp, ctypes.POINTER(kl_kernel_stats), c_int, ctypes.POINTER(c_int)]),
        "kl_launch_count": (ctypes.c_longlong, [vp]),
        "kl_memory": (c_int, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "kl_last_error": (ctypes.c_char_p, [vp]),
        "kl_status_string": (ctypes.c_char_p, [c_int]),
        "kl_measure_peaks": (c_int, [ctypes.POINTER(dbl)] * 3),
        "kl_pairwise_noalloc": (c_int, [c_int, dbl, dbl, vp, i64, vp, i64, vp, i64, vp, i64, c_int, vp]),
        "kl_estimate_bytes": (c_int, [ctypes.POINTER(kl_params), c_int, ctypes.POINTER(i64)]),
        "kl_serve_open": (c_int, [ctypes.POINTER(kl_serve_config), ctypes.POINTER(vp)]),
        "kl_serve_submit": (c_int, [vp, ctypes.POINTER(kl_params), c_int, dbl, i64, vp, vp, i64]),
        "kl_serve_poll": (c_int, [vp, ctypes.POINTER(kl_serve_result), c_int, ctypes.POINTER(c_int), c_int]),
        "kl_serve_get_stats": (c_int, [vp, ctypes.POINTER(kl_serve_stats)]),
        "kl_serve_close": (c_int, [vp]),
        "kl_set_graphs": (c_int, [vp, c_int]),
        "kl_set_shared_sms": (c_int, [vp, c_int]),
        "kl_block_size": (c_int, [vp]),
        "kl_autotune": (c_int, [ctypes.POINTER(kl_params), c_int, dbl, vp, ctypes.c_char_p, ctypes.POINTER(c_int),
                                ctypes.POINTER(dbl)]),
        "kl_sample_size": (i64, [vp]),
        "kl_sample_points": (c_int, [vp, vp]),
        "kl_sample": (c_int, [vp, c_int, vp, vp, i64, vp, i64, c_int, vp, i64]),
        "kl_bounds_checked": (c_int, []),
        "kl_debug_set": (c_int, [vp, c_int, ctypes.c_longlong]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _check(h, rc, allow=(KL_OK,)):
    if rc in allow:
        return rc
    msg = _load().kl_last_error(h)
    raise KLError(rc, (msg or b"").decode() or kl_status_string(rc))


def kl_status_string(status):
    return _load().kl_status_string(int(status)).decode()


def kl_last_error(h=None):
    return (_load().kl_last_error(h) or b"").decode()


def kl_default_params():
    p = kl_params()
    _load().kl_default_params(ctypes.byref(p))
    return p


def params(geometry="cube", degree=2, elems=(4, 4, 4), kernel="gauss", sigma=1.0, L=0.5,
           method="galerkin", precision="fp64", block_k=8, refine=-1, interp_continuity=-2,
           geo=(1.0, 2.0, 1.0), dim=None, max_restarts=0, seed=2101):
    """kl_params from readable names (marshalling helper)."""
    p = kl_default_params()
    elems = tuple(int(e) for e in elems)
    p.dim = len(elems) if dim is None else int(dim)
    p.geometry = GEOMETRIES[geometry]
    for i in range(3):
        p.geo[i] = float(geo[i])
        p.elems[i] = elems[i] if i < len(elems) else 1
    p.degree = int(degree)
    p.kernel = KERNELS[kernel]
    p.sigma = float(sigma)
    p.L = float(L)
    p.method = METHODS[method]
    p.interp_continuity = int(interp_continuity)
    p.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    p.block_k = int(block_k)
    p.refine = int(refine)
    p.max_restarts = int(max_restarts)
    p.seed = int(seed)
    return p


def kl_create(p, stream=None):
    """Returns an opaque handle (ctypes.c_void_p). `stream` is a cudaStream_t
    address, a torch.cuda.Stream, or None (legacy default stream)."""
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    h = ctypes.c_void_p()
    rc = _load().kl_create(ctypes.byref(p), stream, ctypes.byref(h))
    _check(None, rc)
    return h


def kl_destroy(h):
    return _check(h, _load().kl_destroy(h))


def kl_dims(h):
    N, S, T = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(h, _load().kl_dims(h, ctypes.byref(N), ctypes.byref(S), ctypes.byref(T)))
    return N.value, S.value, T.value


def kl_apply_A(h, X, ldx, Y, ldy, k):
    return _check(h, _load().kl_apply_A(h, _ptr(X), ldx, _ptr(Y), ldy, k))


def kl_apply_Zinv(h, X, ldx, Y, ldy, k):
    return _check(h, _load().kl_apply_Zinv(h, _ptr(X), ldx, _ptr(Y), ldy, k))


def kl_apply_Aprime(h, X, ldx, Y, ldy, k):
    return _check(h, _load().kl_apply_Aprime(h, _ptr(X), ldx, _ptr(Y), ldy, k))


def kl_eigs(h, M, tol, lam, V, ldv, v_on_device, resid=None, info=None):
    """lam (and resid) are host buffers: numpy float64 arrays or ctypes
    arrays; V is a host numpy array (v_on_device=0) or a device tensor.
    Returns the status (KL_OK, KL_WARN_COMPLEX or KL_ERR_NOCONV)."""
    def host(a):
        if a is None:
            return None
        if hasattr(a, "ctypes"):
            return a.ctypes.data
        return _ptr(a)
    rc = _load().kl_eigs(h, int(M), float(tol), host(lam), host(V) if not v_on_device else _ptr(V),
                         int(ldv), int(v_on_device), host(resid),
                         ctypes.byref(info) if info is not None else None)
    return _check(h, rc, allow=(KL_OK, KL_WARN_COMPLEX, KL_ERR_NOCONV))


def kl_profile_enable(h, on=True):
    return _check(h, _load().kl_profile_enable(h, int(bool(on))))


def kl_profile_read(h):
    buf = (kl_kernel_stats * 32)()
    n = ctypes.c_int()
    _check(h, _load().kl_profile_read(h, buf, 32, ctypes.byref(n)))
    return {buf[i].name.decode(): dict(launches=buf[i].launches, ms=buf[i].ms, units=buf[i].units)
            for i in range(min(n.value, 32))}


def kl_launch_count(h):
    return int(_load().kl_launch_count(h))


def kl_memory(h):
    a, b = ctypes.c_int64(), ctypes.c_int64()
    _check(h, _load().kl_memory(h, ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def kl_measure_peaks():
    """(fp32 FMA/s, ex2/s, fp64 FMA/s) measured on the current device."""
    a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(None, _load().kl_measure_peaks(ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def kl_pairwise_noalloc(kernel, sigma, L, tgt, T, src, S, X, ldx, Y, ldy, k, stream=None):
    """Y = sigma^2 Gamma(tgt, src) X without device allocation (see kl.h)."""
    if isinstance(kernel, str):
        kernel = KERNELS[kernel]
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    rc = _load().kl_pairwise_noalloc(int(kernel), float(sigma), float(L), _ptr(tgt), int(T), _ptr(src), int(S),
                                     _ptr(X), int(ldx), _ptr(Y), int(ldy), int(k), stream)
    return _check(None, rc)


def kl_estimate_bytes(p, M):
    """Device bytes a handle with params p holds while solving for M pairs
    (host-side estimate, no GPU needed)."""
    b = ctypes.c_int64()
    _check(None, _load().kl_estimate_bytes(ctypes.byref(p), int(M), ctypes.byref(b)))
    return b.value


def kl_serve_open(hbm_budget_bytes=0, max_slots=0, batch_window_us=0):
    cfg = kl_serve_config(int(hbm_budget_bytes), int(max_slots), int(batch_window_us))
    s = ctypes.c_void_p()
    _check(None, _load().kl_serve_open(ctypes.byref(cfg), ctypes.byref(s)))
    return s


def kl_serve_submit(s, p, M, tol, request_id, lambda_out, V_out=None, ldv=0):
    """lambda_out / V_out: host buffers (numpy arrays or addresses) that must
    stay alive until the result has been polled."""
    def addr(x):
        if x is None:
            return None
        if isinstance(x, int):
            return x
        return x.ctypes.data
    return _check(None, _load().kl_serve_submit(s, ctypes.byref(p), int(M), float(tol), int(request_id),
                                                addr(lambda_out), addr(V_out), int(ldv)))


def kl_serve_poll(s, cap=64, wait_ms=0):
    buf = (kl_serve_result * cap)()
    n = ctypes.c_int()
    _check(None, _load().kl_serve_poll(s, buf, int(cap), ctypes.byref(n), int(wait_ms)))
    return [{f[0]: getattr(buf[i], f[0]) for f in kl_serve_result._fields_} for i in range(n.value)]


def kl_serve_get_stats(s):
    st = kl_serve_stats()
    _check(None, _load().kl_serve_get_stats(s, ctypes.byref(st)))
    return {f[0]: getattr(st, f[0]) for f in kl_serve_stats._fields_}


def kl_serve_close(s):
    return _check(None, _load().kl_serve_close(s))


def kl_set_graphs(h, on=True):
    return _check(h, _load().kl_set_graphs(h, int(bool(on))))


def kl_set_shared_sms(h, n):
    """SMs the handle's pairwise product leaves free for other streams."""
    return _check(h, _load().kl_set_shared_sms(h, int(n)))


def kl_block_size(h):
    return int(_load().kl_block_size(h))


def kl_autotune(p, M, tol=0.0, stream=None, cache_path=None):
    """(best block size, [seconds for k = 8, 16, 32]) from timed solves."""
    k = ctypes.c_int()
    secs = (ctypes.c_double * 3)()
    if stream is not None and not isinstance(stream, int):
        stream = stream.cuda_stream
    _check(None, _load().kl_autotune(ctypes.byref(p), int(M), float(tol), stream,
                                     cache_path.encode() if cache_path else None, ctypes.byref(k), secs))
    return k.value, list(secs)


def kl_debug_set(h, what, value):
    """Host-side failure injection and comparison switches for tests (see
    kl.h): what is KL_DEBUG_WAIT_LIMIT, KL_DEBUG_FAIL_ALLOC (h may be None),
    KL_DEBUG_NAN_START or KL_DEBUG_PAIR_DENSE."""
    return _check(h, _load().kl_debug_set(h, int(what), int(value)))


def kl_bounds_checked():
    """True if libkl.so is the bounds-checking build (KL_CHECK_BOUNDS)."""
    return bool(_load().kl_bounds_checked())


def kl_sample_size(h):
    return int(_load().kl_sample_size(h))


def kl_sample_points(h, xyz):
    """xyz: device buffer of 3 * kl_sample_size doubles (x, then y, then z)."""
    return _check(h, _load().kl_sample_points(h, _ptr(xyz)))


def kl_sample(h, M, lam, V, ldv, xi, ldxi, ns, out, ldo):
    """lam: host float64 array (M); V, xi, out: device buffers (see kl.h)."""
    import numpy as _np
    lam = _np.ascontiguousarray(lam, dtype=_np.float64)
    return _check(h, _load().kl_sample(h, int(M), lam.ctypes.data, _ptr(V), int(ldv), _ptr(xi), int(ldxi),
                                       int(ns), _ptr(out), int(ldo)))
