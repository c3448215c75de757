"""Python binding of libtoeplitz_ols.so (the C ABI in include/toeplitz_ols.h): argument marshalling only.

Every step of a solve runs in the library's CUDA kernels. Importing this module loads the shared library and
raises if it is missing (run ``python -m paper_2112_12994_gb300.build`` or ``__graft_entry__.build()``); there
is no CPU fallback.

Host arrays are numpy float64 arrays. Device arrays are anything with a ``data_ptr()`` method (a CUDA torch
tensor) or a plain integer address; their element type must match the call (float64, or float32 for the mixed
step entry points).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtoeplitz_ols.so")

TOLS_OK = 0
TOLS_NOT_CONVERGED = 1
TOLS_ERR_ARG = -1
TOLS_ERR_NONFINITE = -2
TOLS_ERR_OOM = -3
TOLS_ERR_CUDA = -4
TOLS_ERR_DEVICE_TIMEOUT = -5
TOLS_ERR_NO_DEVICE = -6
TOLS_ERR_BUSY = -7
TOLS_MAX_P = 1024
TOLS_NOALLOC_MAX_P = 256

TOLS_FP64 = 0
TOLS_MIXED = 1
TOLS_PRECOND_NONE = 0
TOLS_PRECOND_GRAM_CHOL = 1
TOLS_PRECOND_SAMPLED_QR = 2
TOLS_PRODUCT_AUTO = 0
TOLS_PRODUCT_DIRECT = 1
TOLS_PRODUCT_FFT = 2
TOLS_PRODUCT_FFT4096 = 3
TOLS_PROFILE_CLASSES = 17
PROFILE_CLASS_NAMES = ["pass_f32_store", "pass_f32_lsqr", "pass_f32_necorr", "pass_f32_check", "pass_f32_gram",
                       "pass_f64_store", "pass_f64_lsqr", "pass_f64_necorr", "pass_f64_check", "pass_f64_gram",
                       "precond", "convert_f32", "small",
                       "batch_f64_fft", "batch_f64_direct", "batch_f32_direct", "batch_dspec"]


class tols_config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("device", ctypes.c_int), ("mem_cap_bytes", ctypes.c_size_t),
                ("max_iter", ctypes.c_int), ("max_sweeps", ctypes.c_int), ("precond", ctypes.c_int),
                ("product", ctypes.c_int), ("cuda_stream", ctypes.c_void_p), ("wait_polls", ctypes.c_int)]


class tols_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iters", ctypes.c_int), ("sweeps", ctypes.c_int),
                ("precision_used", ctypes.c_int), ("precond_used", ctypes.c_int), ("product_used", ctypes.c_int),
                ("ne_ratio", ctypes.c_double), ("rnorm", ctypes.c_double), ("bnorm", ctypes.c_double),
                ("anorm_2", ctypes.c_double), ("anorm_f", ctypes.c_double), ("cond_est", ctypes.c_double),
                ("nfft", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class tols_server_config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("device", ctypes.c_int), ("arena_bytes", ctypes.c_size_t),
                ("max_active", ctypes.c_int), ("burst", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("max_sweeps", ctypes.c_int), ("cuda_stream", ctypes.c_void_p)]


class tols_result(ctypes.Structure):
    _fields_ = [("id", ctypes.c_longlong), ("status", ctypes.c_int), ("p", ctypes.c_int),
                ("latency_s", ctypes.c_double), ("info", tols_info)]


class tols_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("active", ctypes.c_int),
                ("queued", ctypes.c_int), ("arena_bytes", ctypes.c_size_t), ("arena_used", ctypes.c_size_t)]


class TolsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2112_12994_gb300.build.build()")
    return ctypes.CDLL(LIB_PATH)


lib = _load()

_P = ctypes.c_void_p
_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.c_int
_LL = ctypes.c_longlong

# symbol table: name -> (restype, argtypes); every entry point of include/toeplitz_ols.h
SIGNATURES = {
    "toeplitz_ols_config_default": (None, [ctypes.POINTER(tols_config)]),
    "toeplitz_ols_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(tols_config)]),
    "toeplitz_ols_destroy": (_I, [_P]),
    "toeplitz_ols_strerror": (ctypes.c_char_p, [_I]),
    "toeplitz_ols_last_error": (ctypes.c_char_p, [_P]),
    "toeplitz_ols_solve": (_I, [_P, _P, _LL, _I, ctypes.c_double, _P, _D, ctypes.POINTER(tols_info)]),
    "toeplitz_ols_solve_device": (_I, [_P, _P, _LL, _I, ctypes.c_double, _P, _D, ctypes.POINTER(tols_info)]),
    "toeplitz_ols_solve_batched": (_I, [_P, _I, _P, _P, _P, ctypes.c_double, _P, _P, _P]),
    "toeplitz_ols_solve_batched_device": (_I, [_P, _I, _P, _P, _P, ctypes.c_double, _P, _P, _P]),
    "toeplitz_ols_pacf": (_I, [_P, _P, _LL, _I, ctypes.c_double, _P, ctypes.POINTER(_I), _P]),
    "toeplitz_ols_stream_open": (_I, [_P, _I, ctypes.c_double, ctypes.POINTER(_I)]),
    "toeplitz_ols_stream_push": (_I, [_P, _I, _P, _LL]),
    "toeplitz_ols_stream_solve": (_I, [_P, _I, _P, _D, ctypes.POINTER(tols_info)]),
    "toeplitz_ols_stream_close": (_I, [_P, _I]),
    "toeplitz_ols_gk_pass": (_I, [_P, _I, _P, _LL, _I, _P, _P, ctypes.c_double, _P, _P, _D]),
    "toeplitz_ols_gk_pass_noalloc": (_I, [_I, _P, _LL, _I, _P, _P, ctypes.c_double, _P, _P, _P, _P]),
    "toeplitz_ols_gram": (_I, [_P, _I, _P, _LL, _I, _P, _P, _D]),
    "toeplitz_ols_preconditioner": (_I, [_P, _I, _P, _LL, _I, _I, _P, ctypes.POINTER(tols_info)]),
    "toeplitz_ols_row_norms": (_I, [_P, _P, _LL, _I, _P, _D]),
    "toeplitz_ols_residual": (_I, [_P, _P, _LL, _I, _P, _P, _D]),
    "toeplitz_ols_leverage_p1": (_I, [_P, _P, _LL, _P]),
    "toeplitz_ols_leverage_step": (_I, [_P, _P, _LL, _I, _P, _P, _P, _P, _D]),
    "toeplitz_ols_lsar": (_I, [_P, _P, _LL, _I, _I, _P, _P, ctypes.POINTER(_I), _P, _P, _P]),
    "toeplitz_ols_rh_lsar": (_I, [_P, _P, _LL, _I, _I, _I, _I, _P, _P, _P, _P, _P, _P, ctypes.POINTER(_I), _P, _P,
                                  _P]),
    "toeplitz_ols_srht": (_I, [_P, _P, _LL, _I, _I, _P, _P, _P]),
    "toeplitz_ols_server_config_default": (None, [ctypes.POINTER(tols_server_config)]),
    "toeplitz_ols_server_create": (_I, [ctypes.POINTER(_P), ctypes.POINTER(tols_server_config)]),
    "toeplitz_ols_server_destroy": (_I, [_P]),
    "toeplitz_ols_server_submit": (_I, [_P, _LL, _P, _LL, _I, ctypes.c_double]),
    "toeplitz_ols_server_step": (_I, [_P, ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "toeplitz_ols_server_poll": (_I, [_P, _P, _P, _I, ctypes.POINTER(_I)]),
    "toeplitz_ols_server_stats": (_I, [_P, ctypes.POINTER(tols_server_stats)]),
    "toeplitz_ols_profile": (_I, [_P, _I]),
    "toeplitz_ols_profile_read": (_I, [_P, _I, ctypes.POINTER(ctypes.c_longlong), _D]),
}

for _name, (_res, _args) in SIGNATURES.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def _ptr(x):
    """Device address of a torch tensor / integer, or host address of a numpy array."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x).__name__}")


def _host_f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _dev(x, count, itemsize, name):
    """Check a device-buffer argument before its address reaches a kernel: a tensor must be contiguous, have
    elements of itemsize bytes and hold at least count of them (raw integer addresses pass unchecked)."""
    if x is None or isinstance(x, int):
        return
    if hasattr(x, "element_size") and x.element_size() != itemsize:
        raise TolsError(TOLS_ERR_ARG, f"{name}: elements of {x.element_size()} bytes, expected {itemsize}")
    if hasattr(x, "is_contiguous") and not x.is_contiguous():
        raise TolsError(TOLS_ERR_ARG, f"{name}: not contiguous")
    if hasattr(x, "numel") and x.numel() < count:
        raise TolsError(TOLS_ERR_ARG, f"{name}: {x.numel()} elements, needs {count}")


def _pass_itemsize(precision):
    return 8 if precision == TOLS_FP64 else 4


def strerror(code: int) -> str:
    return lib.toeplitz_ols_strerror(code).decode()


class Context:
    """Owns a tols_ctx handle (toeplitz_ols_create / toeplitz_ols_destroy)."""

    def __init__(self, precision=TOLS_FP64, device=0, mem_cap_bytes=0, max_iter=0, max_sweeps=0,
                 precond=TOLS_PRECOND_GRAM_CHOL, product=TOLS_PRODUCT_AUTO, cuda_stream=None, wait_polls=0):
        cfg = tols_config()
        lib.toeplitz_ols_config_default(ctypes.byref(cfg))
        cfg.precision, cfg.device, cfg.mem_cap_bytes = precision, device, mem_cap_bytes
        cfg.max_iter, cfg.max_sweeps, cfg.precond, cfg.product = max_iter, max_sweeps, precond, product
        cfg.cuda_stream = cuda_stream
        cfg.wait_polls = wait_polls
        h = ctypes.c_void_p()
        rc = lib.toeplitz_ols_create(ctypes.byref(h), ctypes.byref(cfg))
        if rc != TOLS_OK:
            raise TolsError(rc, "toeplitz_ols_create: " + strerror(rc))
        self.handle = h
        self.config = cfg

    def close(self):
        if getattr(self, "handle", None):
            lib.toeplitz_ols_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def last_error(self) -> str:
        return lib.toeplitz_ols_last_error(self.handle).decode()

    def check(self, rc, what, allow=(TOLS_OK, TOLS_NOT_CONVERGED)):
        if rc not in allow:
            raise TolsError(rc, f"{what}: {strerror(rc)}: {self.last_error()}")
        return rc


def toeplitz_ols_create(**kw) -> Context:
    return Context(**kw)


def toeplitz_ols_destroy(ctx: Context):
    ctx.close()


def toeplitz_ols_solve(ctx: Context, y, p: int, tol: float = 0.0):
    """Host series y -> (phi (p,), rnorm, info dict, status)."""
    y = _host_f64(y)
    phi = np.zeros(p, dtype=np.float64)
    rn = ctypes.c_double()
    info = tols_info()
    rc = lib.toeplitz_ols_solve(ctx.handle, y.ctypes.data, y.size, p, tol, phi.ctypes.data, ctypes.byref(rn),
                                ctypes.byref(info))
    ctx.check(rc, "toeplitz_ols_solve")
    return phi, rn.value, info.as_dict(), rc


def toeplitz_ols_solve_device(ctx: Context, d_y, n: int, p: int, d_phi, tol: float = 0.0):
    """Device series d_y (n float64) -> d_phi (p float64, device); returns (rnorm, info dict, status)."""
    _dev(d_y, n, 8, "d_y")
    _dev(d_phi, p, 8, "d_phi")
    rn = ctypes.c_double()
    info = tols_info()
    rc = lib.toeplitz_ols_solve_device(ctx.handle, _ptr(d_y), n, p, tol, _ptr(d_phi), ctypes.byref(rn),
                                       ctypes.byref(info))
    ctx.check(rc, "toeplitz_ols_solve_device")
    return rn.value, info.as_dict(), rc


def toeplitz_ols_solve_batched(ctx: Context, ys, ps, tol: float = 0.0):
    """List of host series and orders -> (list of phi, rnorm array, list of info dicts, worst status)."""
    count = len(ys)
    ys = [_host_f64(y) for y in ys]
    phis = [np.zeros(int(p), dtype=np.float64) for p in ps]
    yp = (ctypes.c_void_p * count)(*[y.ctypes.data for y in ys])
    pp = (ctypes.c_void_p * count)(*[f.ctypes.data for f in phis])
    ns = np.array([y.size for y in ys], dtype=np.int64)
    pv = np.array(ps, dtype=np.int32)
    rn = np.zeros(count, dtype=np.float64)
    infos = (tols_info * count)()
    rc = lib.toeplitz_ols_solve_batched(ctx.handle, count, ctypes.cast(yp, _P), ns.ctypes.data, pv.ctypes.data, tol,
                                        ctypes.cast(pp, _P), rn.ctypes.data, ctypes.cast(infos, _P))
    ctx.check(rc, "toeplitz_ols_solve_batched")
    return phis, rn, [i.as_dict() for i in infos], rc


def toeplitz_ols_solve_batched_device(ctx: Context, d_ys, ps, d_phi, tol: float = 0.0):
    """Device series (list of CUDA tensors / addresses) -> coefficients packed in d_phi (device, sum(ps));
    returns (rnorm array, list of info dicts, worst status)."""
    count = len(d_ys)
    for y in d_ys:
        _dev(y, 0, 8, "d_ys[k]")
    _dev(d_phi, int(sum(int(q) for q in ps)), 8, "d_phi")
    yp = (ctypes.c_void_p * count)(*[_ptr(y) for y in d_ys])
    ns = np.array([int(y.numel()) if hasattr(y, "numel") else 0 for y in d_ys], dtype=np.int64)
    pv = np.array(ps, dtype=np.int32)
    rn = np.zeros(count, dtype=np.float64)
    infos = (tols_info * count)()
    rc = lib.toeplitz_ols_solve_batched_device(ctx.handle, count, ctypes.cast(yp, _P), ns.ctypes.data,
                                               pv.ctypes.data, tol, _ptr(d_phi), rn.ctypes.data,
                                               ctypes.cast(infos, _P))
    ctx.check(rc, "toeplitz_ols_solve_batched_device")
    return rn, [i.as_dict() for i in infos], rc


def toeplitz_ols_pacf(ctx: Context, y, h_max: int, tol: float = 0.0):
    """Host series, largest lag -> (tau array of h_max PACF estimates, estimated order, list of info dicts, worst
    status). tau[h-1] is the last coefficient of the AR(h) fit."""
    y = _host_f64(y)
    tau = np.zeros(int(h_max), dtype=np.float64)
    order = ctypes.c_int(0)
    infos = (tols_info * int(h_max))()
    rc = lib.toeplitz_ols_pacf(ctx.handle, y.ctypes.data, y.size, int(h_max), tol, tau.ctypes.data,
                               ctypes.byref(order), ctypes.cast(infos, _P))
    ctx.check(rc, "toeplitz_ols_pacf")
    return tau, order.value, [i.as_dict() for i in infos], rc


def toeplitz_ols_stream_open(ctx: Context, p: int, tol: float = 0.0) -> int:
    h = ctypes.c_int()
    ctx.check(lib.toeplitz_ols_stream_open(ctx.handle, p, tol, ctypes.byref(h)), "toeplitz_ols_stream_open")
    return h.value


def toeplitz_ols_stream_push(ctx: Context, handle: int, chunk):
    chunk = _host_f64(chunk)
    ctx.check(lib.toeplitz_ols_stream_push(ctx.handle, handle, chunk.ctypes.data, chunk.size),
              "toeplitz_ols_stream_push")


def toeplitz_ols_stream_solve(ctx: Context, handle: int, p: int):
    phi = np.zeros(p, dtype=np.float64)
    rn = ctypes.c_double()
    info = tols_info()
    rc = lib.toeplitz_ols_stream_solve(ctx.handle, handle, phi.ctypes.data, ctypes.byref(rn), ctypes.byref(info))
    ctx.check(rc, "toeplitz_ols_stream_solve")
    return phi, rn.value, info.as_dict(), rc


def toeplitz_ols_stream_close(ctx: Context, handle: int):
    ctx.check(lib.toeplitz_ols_stream_close(ctx.handle, handle), "toeplitz_ols_stream_close")


def _check_pass_args(precision, d_y, n, p, d_v, d_u_old, d_u_new, d_xtu):
    es = _pass_itemsize(precision)
    _dev(d_y, n, es, "d_y")
    _dev(d_v, p, 8, "d_v")
    _dev(d_u_old, n - p, es, "d_u_old")
    _dev(d_u_new, n - p, es, "d_u_new")
    _dev(d_xtu, p, 8, "d_xtu")


def toeplitz_ols_gk_pass(ctx: Context, precision: int, d_y, n: int, p: int, d_v, d_u_old, c: float, d_u_new, d_xtu):
    """u_new = X v - c u_old, X^T u_new -> d_xtu; returns ||u_new||^2 (device buffers)."""
    _check_pass_args(precision, d_y, n, p, d_v, d_u_old, d_u_new, d_xtu)
    n2 = ctypes.c_double()
    ctx.check(lib.toeplitz_ols_gk_pass(ctx.handle, precision, _ptr(d_y), n, p, _ptr(d_v), _ptr(d_u_old), c,
                                       _ptr(d_u_new), _ptr(d_xtu), ctypes.byref(n2)), "toeplitz_ols_gk_pass")
    return n2.value


def toeplitz_ols_gk_pass_noalloc(precision: int, d_y, n: int, p: int, d_v, d_u_old, c: float, d_u_new, d_xtu,
                                 d_unorm2, stream=None) -> int:
    """The allocation-free fused pass (no context): enqueues on `stream` (a cudaStream_t handle or None) and
    returns the status code without waiting; ||u_new||^2 goes to the device scalar d_unorm2."""
    _check_pass_args(precision, d_y, n, p, d_v, d_u_old, d_u_new, d_xtu)
    _dev(d_unorm2, 1, 8, "d_unorm2")
    return lib.toeplitz_ols_gk_pass_noalloc(precision, _ptr(d_y), n, p, _ptr(d_v), _ptr(d_u_old), c, _ptr(d_u_new),
                                            _ptr(d_xtu), _ptr(d_unorm2), stream)


def toeplitz_ols_gram(ctx: Context, precision: int, d_y, n: int, p: int, d_G, d_h):
    _dev(d_y, n, 8, "d_y")
    _dev(d_G, p * p, 8, "d_G")
    _dev(d_h, p, 8, "d_h")
    b2 = ctypes.c_double()
    ctx.check(lib.toeplitz_ols_gram(ctx.handle, precision, _ptr(d_y), n, p, _ptr(d_G), _ptr(d_h), ctypes.byref(b2)),
              "toeplitz_ols_gram")
    return b2.value


def toeplitz_ols_preconditioner(ctx: Context, precision: int, d_y, n: int, p: int, kind: int, d_M):
    """M = R^{-1} (p x p, row-major, device) of the solver's preconditioner; returns (info dict, status)."""
    _dev(d_y, n, 8, "d_y")
    _dev(d_M, p * p, 8, "d_M")
    info = tols_info()
    rc = lib.toeplitz_ols_preconditioner(ctx.handle, precision, _ptr(d_y), n, p, kind, _ptr(d_M), ctypes.byref(info))
    ctx.check(rc, "toeplitz_ols_preconditioner")
    return info.as_dict(), rc


def toeplitz_ols_row_norms(ctx: Context, d_y, n: int, p: int, d_rn2=None):
    _dev(d_y, n, 8, "d_y")
    _dev(d_rn2, n - p, 8, "d_rn2")
    f = ctypes.c_double()
    ctx.check(lib.toeplitz_ols_row_norms(ctx.handle, _ptr(d_y), n, p, _ptr(d_rn2), ctypes.byref(f)),
              "toeplitz_ols_row_norms")
    return f.value


def toeplitz_ols_residual(ctx: Context, d_y, n: int, p: int, d_phi, d_g):
    _dev(d_y, n, 8, "d_y")
    _dev(d_phi, p, 8, "d_phi")
    _dev(d_g, p, 8, "d_g")
    rn = ctypes.c_double()
    ctx.check(lib.toeplitz_ols_residual(ctx.handle, _ptr(d_y), n, p, _ptr(d_phi), _ptr(d_g), ctypes.byref(rn)),
              "toeplitz_ols_residual")
    return rn.value


def toeplitz_ols_leverage_p1(ctx: Context, d_y, n: int, d_lev):
    _dev(d_y, n, 8, "d_y")
    _dev(d_lev, n - 1, 8, "d_lev")
    ctx.check(lib.toeplitz_ols_leverage_p1(ctx.handle, _ptr(d_y), n, _ptr(d_lev)), "toeplitz_ols_leverage_p1")


def toeplitz_ols_leverage_step(ctx: Context, d_y, n: int, p: int, d_phi_hat, d_lev_prev, d_lev, d_pi=None):
    _dev(d_y, n, 8, "d_y")
    _dev(d_phi_hat, p - 1, 8, "d_phi_hat")
    for name, buf in (("d_lev_prev", d_lev_prev), ("d_lev", d_lev), ("d_pi", d_pi)):
        _dev(buf, n - p, 8, name)
    rr = ctypes.c_double()
    ctx.check(lib.toeplitz_ols_leverage_step(ctx.handle, _ptr(d_y), n, p, _ptr(d_phi_hat), _ptr(d_lev_prev),
                                             _ptr(d_lev), _ptr(d_pi), ctypes.byref(rr)), "toeplitz_ols_leverage_step")
    return rr.value


def toeplitz_ols_lsar(ctx: Context, d_y, n: int, p_bar: int, c: int, d_unif, d_rows=None, d_phi_all=None):
    """Algorithm LSAR on a device series with device uniforms (p_bar x c) -> (tau array of p_bar PACF estimates,
    estimated order, phi_hat at that order (p_bar doubles, zero-padded), status)."""
    _dev(d_y, n, 8, "d_y")
    _dev(d_unif, p_bar * c, 8, "d_unif")
    _dev(d_rows, p_bar * c, 8, "d_rows")
    _dev(d_phi_all, p_bar * p_bar, 8, "d_phi_all")
    tau = np.zeros(int(p_bar), dtype=np.float64)
    phi = np.zeros(int(p_bar), dtype=np.float64)
    order = ctypes.c_int(0)
    rc = lib.toeplitz_ols_lsar(ctx.handle, _ptr(d_y), int(n), int(p_bar), int(c), _ptr(d_unif), tau.ctypes.data,
                               ctypes.byref(order), phi.ctypes.data, _ptr(d_rows), _ptr(d_phi_all))
    ctx.check(rc, "toeplitz_ols_lsar")
    return tau, order.value, phi, rc


def toeplitz_ols_rh_lsar(ctx: Context, d_y, n: int, p_bar: int, c: int, k: int, keep, d_sketch, d_rh_unif, d_unif,
                         d_scores=None, d_rows=None):
    """The Repeated Halving variant of LSAR. keep: list of host integer arrays, level j's kept positions (the
    halvings, from m = n - p_bar rows); d_sketch: one device array holding the k x rows sketches of every level
    in turn (row-major); d_rh_unif: device, levels x c; d_unif: device, p_bar x c. Returns (tau, order, phi,
    status)."""
    levels = len(keep)
    m = int(n) - int(p_bar)
    sizes = np.empty(levels + 1, dtype=np.int64)
    sizes[0] = m
    for j, kj in enumerate(keep):
        sizes[j + 1] = len(kj)
    flat = np.ascontiguousarray(np.concatenate([np.asarray(kj, dtype=np.int64) for kj in keep]) if levels else
                                np.zeros(0, dtype=np.int64))
    deep = int(sizes[-1])
    rows_b = [deep if j == levels - 1 else int(c) for j in range(levels)]
    _dev(d_y, n, 8, "d_y")
    _dev(d_sketch, k * sum(rows_b), 8, "d_sketch")
    _dev(d_rh_unif, levels * c, 8, "d_rh_unif")
    _dev(d_unif, p_bar * c, 8, "d_unif")
    _dev(d_scores, m, 8, "d_scores")
    _dev(d_rows, p_bar * c, 8, "d_rows")
    tau = np.zeros(int(p_bar), dtype=np.float64)
    phi = np.zeros(int(p_bar), dtype=np.float64)
    order = ctypes.c_int(0)
    rc = lib.toeplitz_ols_rh_lsar(ctx.handle, _ptr(d_y), int(n), int(p_bar), int(c), int(k), int(levels),
                                  sizes.ctypes.data, flat.ctypes.data, _ptr(d_sketch), _ptr(d_rh_unif), _ptr(d_unif),
                                  tau.ctypes.data, ctypes.byref(order), phi.ctypes.data, _ptr(d_scores), _ptr(d_rows))
    ctx.check(rc, "toeplitz_ols_rh_lsar")
    return tau, order.value, phi, rc


def toeplitz_ols_srht(ctx: Context, d_y, n: int, p: int, d_signs, d_rows, d_phi):
    """Algorithm SRHT for the order-p problem: device series, signs (m2 = next power of two >= n - p of them),
    c = len(d_rows) sampled row indices (int64) -> d_phi (p doubles, device); returns the status."""
    m = int(n) - int(p)
    m2 = 1 << max(0, (m - 1).bit_length())
    c = int(d_rows.numel()) if hasattr(d_rows, "numel") else 0
    _dev(d_y, n, 8, "d_y")
    _dev(d_signs, m2, 8, "d_signs")
    _dev(d_rows, c, 8, "d_rows")
    _dev(d_phi, p, 8, "d_phi")
    rc = lib.toeplitz_ols_srht(ctx.handle, _ptr(d_y), int(n), int(p), c, _ptr(d_signs), _ptr(d_rows), _ptr(d_phi))
    ctx.check(rc, "toeplitz_ols_srht")
    return rc


def toeplitz_ols_profile(ctx: Context, enable: bool):
    ctx.check(lib.toeplitz_ols_profile(ctx.handle, int(bool(enable))), "toeplitz_ols_profile")


def toeplitz_ols_profile_read(ctx: Context, kind: int):
    """(launches, total_ms) of one kernel class; kind = -1 gives (all launches, 0.0)."""
    n = ctypes.c_longlong()
    ms = ctypes.c_double()
    ctx.check(lib.toeplitz_ols_profile_read(ctx.handle, kind, ctypes.byref(n), ctypes.byref(ms)),
              "toeplitz_ols_profile_read")
    return n.value, ms.value


class Server:
    """A continuous-batching server (toeplitz_ols_server_*): submit fit requests, step, poll results."""

    def __init__(self, precision=TOLS_MIXED, device=0, arena_bytes=0, max_active=1024, burst=4, max_iter=0,
                 max_sweeps=0, cuda_stream=None):
        cfg = tols_server_config()
        lib.toeplitz_ols_server_config_default(ctypes.byref(cfg))
        cfg.precision, cfg.device, cfg.arena_bytes = precision, device, arena_bytes
        cfg.max_active, cfg.burst, cfg.max_iter, cfg.max_sweeps = max_active, burst, max_iter, max_sweeps
        cfg.cuda_stream = cuda_stream
        h = ctypes.c_void_p()
        rc = lib.toeplitz_ols_server_create(ctypes.byref(h), ctypes.byref(cfg))
        if rc != TOLS_OK:
            raise TolsError(rc, "toeplitz_ols_server_create: " + strerror(rc))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib.toeplitz_ols_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def submit(self, rid: int, y, p: int, tol: float = 0.0) -> int:
        y = _host_f64(y)
        return lib.toeplitz_ols_server_submit(self.handle, rid, y.ctypes.data, y.size, p, tol)

    def step(self):
        a, q = ctypes.c_int(), ctypes.c_int()
        rc = lib.toeplitz_ols_server_step(self.handle, ctypes.byref(a), ctypes.byref(q))
        if rc != TOLS_OK:
            raise TolsError(rc, "toeplitz_ols_server_step: " + strerror(rc))
        return a.value, q.value

    def poll(self, max_results: int = 1024):
        out = (tols_result * max_results)()
        phi = np.zeros(max_results * TOLS_MAX_P)
        got = ctypes.c_int()
        rc = lib.toeplitz_ols_server_poll(self.handle, ctypes.cast(out, ctypes.c_void_p), phi.ctypes.data,
                                          max_results, ctypes.byref(got))
        if rc != TOLS_OK:
            raise TolsError(rc, "toeplitz_ols_server_poll: " + strerror(rc))
        res = []
        for i in range(got.value):
            r = out[i]
            res.append({"id": r.id, "status": r.status, "p": r.p, "latency_s": r.latency_s,
                        "info": r.info.as_dict(), "phi": phi[i * TOLS_MAX_P: i * TOLS_MAX_P + r.p].copy()})
        return res

    def stats(self):
        st = tols_server_stats()
        lib.toeplitz_ols_server_stats(self.handle, ctypes.byref(st))
        return {k: getattr(st, k) for k, _ in st._fields_}

    def run_until_idle(self, max_steps: int = 100000):
        results = []
        for _ in range(max_steps):
            active, queued = self.step()
            results += self.poll()
            if active == 0 and queued == 0:
                break
        return results
