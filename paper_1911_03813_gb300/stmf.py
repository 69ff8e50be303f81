"""Python binding of libstmf (include/stmf.h): argument marshalling only.

Every step of the evaluation runs in the library's CUDA kernels; this module passes torch device
pointers, sizes and the current CUDA stream across the C ABI and raises StmfError on a non-zero
status. There is no other implementation behind these names: if libstmf.so is missing or fails
to load, every call raises.
"""

import ctypes
import os
import threading

import torch

from . import _build

STMF_F64, STMF_F32, STMF_BF16, STMF_E4M3 = 0, 1, 2, 3
SERVER_PASS_TILES = 128  # STMF_SERVER_PASS_TILES of include/stmf.h
_TORCH_DTYPE = {
    torch.float64: STMF_F64,
    torch.float32: STMF_F32,
    torch.bfloat16: STMF_BF16,
    torch.float8_e4m3fn: STMF_E4M3,
}
_NAME_DTYPE = {"f64": STMF_F64, "f32": STMF_F32, "bf16": STMF_BF16, "e4m3": STMF_E4M3}


class StmfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (status_string(status), msg))
        self.status = status


class Samples(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("scale", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("p", ctypes.c_int64), ("ld", ctypes.c_int64), ("dtype", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_lib = None
_lock = threading.Lock()


def lib():
    """Load libstmf.so (built in-tree by _build.build()); raise if it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libstmf.so is not built: run paper_1911_03813_gb300._build.build() "
                               "(or __graft_entry__.build()) first")
        L = ctypes.CDLL(_build.LIB)
        vp, i32, i64, dp = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p
        L.stmf_version.restype = ctypes.c_int
        L.stmf_status_string.restype = ctypes.c_char_p
        L.stmf_status_string.argtypes = [ctypes.c_int]
        L.stmf_create.argtypes = [ctypes.c_int, ctypes.POINTER(vp)]
        L.stmf_destroy.argtypes = [vp]
        L.stmf_last_error.restype = ctypes.c_char_p
        L.stmf_last_error.argtypes = [vp]
        L.stmf_reserve.argtypes = [vp, ctypes.POINTER(Samples), i64]
        L.stmf_device_status.argtypes = [vp, vp, ctypes.POINTER(i32)]
        L.stmf_fg.argtypes = [vp, ctypes.POINTER(Samples), dp, i32, i64, dp, dp, dp, dp, dp, dp,
                              vp]
        L.stmf_norm_x.argtypes = [vp, ctypes.POINTER(Samples), dp, i32, dp, vp]
        L.stmf_norm_x_method.argtypes = [vp, ctypes.POINTER(Samples), dp, i32, i32, dp, vp]
        L.stmf_norm_x_method.restype = ctypes.c_int
        L.stmf_profile_enable.argtypes = [vp, i32]
        L.stmf_set_pass_tiles.argtypes = [vp, i32]
        L.stmf_set_pass_tiles.restype = ctypes.c_int
        L.stmf_profile_read.argtypes = [vp, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(i64)]
        for name in ("stmf_create", "stmf_destroy", "stmf_reserve", "stmf_device_status",
                     "stmf_fg", "stmf_norm_x", "stmf_profile_enable", "stmf_profile_read"):
            getattr(L, name).restype = ctypes.c_int
        _declare_extras(L)
        _lib = L
    return _lib


_extra_declarers = []


def _declare_extras(L):
    for fn in _extra_declarers:
        fn(L)


def status_string(status):
    try:
        return lib().stmf_status_string(int(status)).decode()
    except Exception:  # pragma: no cover
        return "status %d" % status


class Context:
    """An stmf context on one CUDA device (owns the library's workspace)."""

    def __init__(self, device=None):
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        h = ctypes.c_void_p()
        st = lib().stmf_create(self.device, ctypes.byref(h))
        if st != 0:
            raise StmfError(st, "stmf_create(%d) failed" % self.device)
        self.handle = h

    def check(self, st, what):
        if st != 0:
            msg = lib().stmf_last_error(self.handle)
            raise StmfError(st, "%s: %s" % (what, msg.decode() if msg else ""))

    def set_pass_tiles(self, min_tiles):
        """stmf_set_pass_tiles: each CTA of this context's tensor-core passes takes at least
        min_tiles tiles of 128 samples (1: one CTA per SM; the server's slots use
        SERVER_PASS_TILES)."""
        self.check(lib().stmf_set_pass_tiles(self.handle, int(min_tiles)), "stmf_set_pass_tiles")

    def device_status(self, stream=None):
        out = ctypes.c_int32()
        self.check(lib().stmf_device_status(self.handle, _stream(stream), ctypes.byref(out)),
                   "stmf_device_status")
        return out.value

    def close(self):
        if getattr(self, "handle", None):
            lib().stmf_destroy(self.handle)
            self.handle = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


_contexts = {}


def default_context(device=None):
    if device is None:
        device = torch.cuda.current_device()
    ctx = _contexts.get(device)
    if ctx is None:
        ctx = Context(device)
        _contexts[device] = ctx
    return ctx


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_f64(t, shape, name):
    if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
        raise ValueError("%s must be a contiguous CUDA float64 tensor" % name)
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(t.shape), tuple(shape)))


def as_samples(V, n=None, scale=None):
    """Build the stmf_samples descriptor of a p x ld CUDA tensor (row l = sample l) whose first n
    columns hold the samples. V may also be a dict as returned by inputs.to_storage. Returns
    (descriptor, keep-alive tuple)."""
    if isinstance(V, dict):
        n = V["n"]
        scale = V.get("scale")
        V = V["data"]
    if V.dim() != 2 or not V.is_cuda:
        raise ValueError("V must be a 2-D CUDA tensor (p x ld)")
    if V.stride(1) != 1:
        raise ValueError("V rows must be contiguous")
    dt = _TORCH_DTYPE.get(V.dtype)
    if dt is None:
        raise ValueError("unsupported sample dtype %s" % V.dtype)
    if n is None:
        n = V.shape[1]
    desc = Samples(V.data_ptr(), scale.data_ptr() if scale is not None else None, int(n),
                   int(V.shape[0]), int(V.stride(0)), dt, 0)
    return desc, (V, scale)


def _check_model_args(desc, nu, lam, A, alpha, out):
    """Validate the model arguments shared by fg() and fg_noalloc() and return the output
    tensors (f (1,), g_lambda (r,), G_A (n, r) column-major), allocating them unless given."""
    n, p = desc.n, desc.p
    r = lam.shape[0]
    _check_f64(lam, (r,), "lambda")
    if A.dtype != torch.float64 or not A.is_cuda or tuple(A.shape) != (n, r):
        raise ValueError("A must be an (n, r) CUDA float64 tensor")
    if not ((A.stride(0) == 1 or n == 1) and (A.stride(1) == n or r == 1)):
        raise ValueError("A must be column-major (A.stride() == (1, n))")
    if nu is not None:
        _check_f64(nu, (p,), "nu")
    if alpha is not None:
        _check_f64(alpha, (1,), "alpha")
    if out is None:
        f = torch.empty(1, dtype=torch.float64, device=lam.device)
        gl = torch.empty(r, dtype=torch.float64, device=lam.device)
        GA = torch.empty((r, n), dtype=torch.float64, device=lam.device).T
    else:
        f, gl, GA = out
        _check_f64(f, (1,), "f")
        _check_f64(gl, (r,), "g_lambda")
        if (GA.dtype != torch.float64 or not GA.is_cuda or tuple(GA.shape) != (n, r)
                or not ((GA.stride(0) == 1 or n == 1) and (GA.stride(1) == n or r == 1))):
            raise ValueError("G_A must be an (n, r) column-major CUDA float64 tensor")
    return f, gl, GA


def fg(V, nu, d, lam, A, alpha=None, out=None, stream=None, ctx=None):
    """f, g_lambda, G_A of Alg. 2 (stmf_fg). lam: (r,) float64 CUDA; A: (n, r) float64 CUDA in
    column-major order (pass A as a Fortran-ordered view, e.g. At.T for At of shape (r, n)).
    nu: (p,) float64 CUDA or None (1/p). alpha: (1,) float64 CUDA or None (0).
    Returns device tensors (f (1,), g_lambda (r,), G_A as an (n, r) column-major view)."""
    ctx = ctx or default_context()
    desc, keep = as_samples(V)
    r = lam.shape[0]
    f, gl, GA = _check_model_args(desc, nu, lam, A, alpha, out)
    st = lib().stmf_fg(ctx.handle, ctypes.byref(desc), _ptr(nu), int(d), int(r), _ptr(lam),
                       _ptr(A), _ptr(alpha), _ptr(f), _ptr(gl), _ptr(GA), _stream(stream))
    ctx.check(st, "stmf_fg")
    del keep
    return f, gl, GA


NORM_X_METHODS = {"auto": 0, "gram": 1, "compressed": 2}


def norm_x(V, nu, d, out=None, stream=None, ctx=None, method="auto"):
    """alpha = ||X||^2 (stmf_norm_x_method): method "gram" = nu^T (V^T V)^d nu, "compressed" =
    from the distinct entries of the symmetric X, "auto" = the cheaper. Returns a (1,) float64
    CUDA tensor."""
    ctx = ctx or default_context()
    desc, keep = as_samples(V)
    if nu is not None:
        _check_f64(nu, (desc.p,), "nu")
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=torch.device("cuda", ctx.device))
    st = lib().stmf_norm_x_method(ctx.handle, ctypes.byref(desc), _ptr(nu), int(d),
                                  NORM_X_METHODS[method], _ptr(out), _stream(stream))
    ctx.check(st, "stmf_norm_x_method")
    del keep
    return out


def reserve(V, r, ctx=None):
    ctx = ctx or default_context()
    desc, keep = as_samples(V)
    ctx.check(lib().stmf_reserve(ctx.handle, ctypes.byref(desc), int(r)), "stmf_reserve")


def profile_enable(enable, ctx=None):
    """Record CUDA events around each fused pass of stmf_fg (benchmark timing)."""
    ctx = ctx or default_context()
    ctx.check(lib().stmf_profile_enable(ctx.handle, 1 if enable else 0), "stmf_profile_enable")


def profile_read(ctx=None):
    """(total pass milliseconds, number of passes) since the last read."""
    ctx = ctx or default_context()
    tot = ctypes.c_double()
    cnt = ctypes.c_int64()
    ctx.check(lib().stmf_profile_read(ctx.handle, ctypes.byref(tot), ctypes.byref(cnt)),
              "stmf_profile_read")
    return tot.value, cnt.value


def _declare_noalloc(L):
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.stmf_fg_noalloc.argtypes = [ctypes.POINTER(Samples), vp, i32, i64, vp, vp, vp, vp, vp, vp,
                                  vp, vp]
    L.stmf_fg_noalloc.restype = ctypes.c_int


_extra_declarers.append(_declare_noalloc)


def fg_noalloc(V, nu, d, lam, A, alpha=None, out=None, status=None, stream=None):
    """stmf_fg_noalloc: the same evaluation as fg(), for callers that cannot allocate device
    memory; the library uses a fixed scratch array in its device globals instead of a context
    workspace. Calls on one device share that array, so calls that overlap on the GPU race.
    Output tensors (f, g_lambda, G_A) may be passed in `out` so that the call itself allocates
    nothing; `status` is an optional (1,) int32 CUDA tensor that receives device-side errors
    (the call does not clear it). Whenever a device-side error is recorded (in `status` or, when
    it is None, in a word of the scratch), f, g_lambda and G_A come back as NaN."""
    desc, keep = as_samples(V)
    r = lam.shape[0]
    f, gl, GA = _check_model_args(desc, nu, lam, A, alpha, out)
    if status is not None and (status.dtype != torch.int32 or not status.is_cuda
                               or tuple(status.shape) != (1,)):
        raise ValueError("status must be a (1,) int32 CUDA tensor")
    st = lib().stmf_fg_noalloc(ctypes.byref(desc), _ptr(nu), int(d), int(r), _ptr(lam), _ptr(A),
                               _ptr(alpha), _ptr(f), _ptr(gl), _ptr(GA), _ptr(status),
                               _stream(stream))
    if st != 0:
        raise StmfError(st, "stmf_fg_noalloc")
    del keep
    return f, gl, GA


class FitOpts(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int32), ("max_ls", ctypes.c_int32), ("pgtol", ctypes.c_double),
                ("factr", ctypes.c_double), ("max_iters", ctypes.c_int64),
                ("max_evals", ctypes.c_int64), ("alpha_mode", ctypes.c_int32),
                ("chunk", ctypes.c_int32)]


class FitResult(ctypes.Structure):
    _fields_ = [("f", ctypes.c_double), ("alpha", ctypes.c_double), ("g_inf", ctypes.c_double),
                ("iters", ctypes.c_int64), ("evals", ctypes.c_int64),
                ("stop_reason", ctypes.c_int32), ("status", ctypes.c_int32)]


STOP_REASONS = {0: "running", 1: "pgtol", 2: "factr", 3: "max_iters", 4: "max_evals",
                5: "line search failed", 6: "non-finite"}


def _declare_fit(L):
    vp = ctypes.c_void_p
    L.stmf_fit_default_opts.argtypes = [ctypes.POINTER(FitOpts)]
    L.stmf_fit_default_opts.restype = ctypes.c_int
    L.stmf_fit.argtypes = [vp, ctypes.POINTER(Samples), vp, ctypes.c_int32, ctypes.c_int64,
                           ctypes.POINTER(FitOpts), vp, vp, ctypes.POINTER(FitResult), vp]
    L.stmf_fit.restype = ctypes.c_int


_extra_declarers.append(_declare_fit)


def fit_options(**kw):
    """stmf_fit_opts with the library defaults, overridden by keyword arguments."""
    o = FitOpts()
    lib().stmf_fit_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def fit(V, nu, d, lam, A, opts=None, stream=None, ctx=None, **kw):
    """stmf_fit: on-device L-BFGS from the start (lam, A); lam (r,) and A (n, r, column-major)
    are CUDA float64 tensors updated in place with the final iterate. Returns a dict."""
    ctx = ctx or default_context()
    desc, keep = as_samples(V)
    n, r = desc.n, lam.shape[0]
    _check_f64(lam, (r,), "lambda")
    if A.dtype != torch.float64 or not A.is_cuda or tuple(A.shape) != (n, r):
        raise ValueError("A must be an (n, r) CUDA float64 tensor")
    if not ((A.stride(0) == 1 or n == 1) and (A.stride(1) == n or r == 1)):
        raise ValueError("A must be column-major (A.stride() == (1, n))")
    if nu is not None:
        _check_f64(nu, (desc.p,), "nu")
    o = opts if opts is not None else fit_options(**kw)
    res = FitResult()
    st = lib().stmf_fit(ctx.handle, ctypes.byref(desc), _ptr(nu), int(d), int(r), ctypes.byref(o),
                        _ptr(lam), _ptr(A), ctypes.byref(res), _stream(stream))
    ctx.check(st, "stmf_fit")
    del keep
    return dict(f=res.f, alpha=res.alpha, g_inf=res.g_inf, iters=res.iters, evals=res.evals,
                stop=res.stop_reason, stop_name=STOP_REASONS.get(res.stop_reason, "?"),
                status=res.status)


class ServerConfig(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_fits", ctypes.c_int32), ("n_max", ctypes.c_int32),
                ("r_max", ctypes.c_int32), ("m_max", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("mem_budget", ctypes.c_size_t)]


class Request(ctypes.Structure):
    _fields_ = [("V", Samples), ("V_on_host", ctypes.c_int32), ("d", ctypes.c_int32),
                ("r", ctypes.c_int64), ("n_starts", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("nu", ctypes.c_void_p), ("x0", ctypes.c_void_p), ("lambda_out", ctypes.c_void_p),
                ("A_out", ctypes.c_void_p), ("opts", FitOpts)]


class RequestResult(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("best_start", ctypes.c_int32), ("best", FitResult),
                ("total_evals", ctypes.c_int64), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("footprint", ctypes.c_size_t)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("admitted", ctypes.c_int64),
                ("completed", ctypes.c_int64), ("cancelled", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("active_fits", ctypes.c_int32),
                ("queued", ctypes.c_int32), ("bytes_in_use", ctypes.c_size_t),
                ("peak_bytes_in_use", ctypes.c_size_t), ("slot_bytes", ctypes.c_size_t),
                ("now", ctypes.c_double), ("peak_active_fits", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


def _declare_server(L):
    vp = ctypes.c_void_p
    L.stmf_server_create.argtypes = [ctypes.POINTER(ServerConfig), ctypes.POINTER(vp)]
    L.stmf_server_destroy.argtypes = [vp]
    L.stmf_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
    L.stmf_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(RequestResult), ctypes.c_int32]
    L.stmf_cancel.argtypes = [vp, ctypes.c_uint64]
    L.stmf_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
    for name in ("stmf_server_create", "stmf_server_destroy", "stmf_submit", "stmf_poll",
                 "stmf_cancel", "stmf_server_get_stats"):
        getattr(L, name).restype = ctypes.c_int


_extra_declarers.append(_declare_server)


class Server:
    """Continuously batched fits (stmf_server_*). Requests carry samples in host memory (numpy
    storage arrays, copied to the device at admission) or on the device (torch tensors)."""

    def __init__(self, device=0, max_fits=16, n_max=128, r_max=16, m_max=5, mem_budget=8 << 30):
        cfg = ServerConfig(int(device), int(max_fits), int(n_max), int(r_max), int(m_max), 0,
                           int(mem_budget))
        h = ctypes.c_void_p()
        st = lib().stmf_server_create(ctypes.byref(cfg), ctypes.byref(h))
        if st != 0:
            raise StmfError(st, "stmf_server_create")
        self.handle = h
        self._keep = {}

    def submit(self, V, d, x0, nu=None, lam_out=None, A_out=None, opts=None, **kw):
        """V: dict with host 'data' (numpy p x ld), optional 'scale', 'n', 'dtype' name; or a
        device storage dict (torch). x0: host float64 array (n_starts, r + n r), each
        [lambda; A column-major]. Returns a ticket."""
        import numpy as np
        x0 = np.ascontiguousarray(x0, dtype=np.float64)
        if x0.ndim == 1:
            x0 = x0[None, :]
        data = V["data"]
        on_host = not (hasattr(data, "is_cuda") and data.is_cuda)
        if on_host:
            arr = np.ascontiguousarray(data)
            scale = V.get("scale")
            if scale is not None:
                scale = np.ascontiguousarray(scale, dtype=np.float32)
            desc = Samples(arr.ctypes.data, scale.ctypes.data if scale is not None else None,
                           int(V["n"]), int(arr.shape[0]), int(arr.shape[1]),
                           _NAME_DTYPE[V["dtype"]], 0)
            keep = (arr, scale)
        else:
            desc, keep = as_samples(V)
        n = desc.n
        r = (x0.shape[1]) // (n + 1)
        o = opts if opts is not None else fit_options(**kw)
        req = Request(desc, 1 if on_host else 0, int(d), int(r), int(x0.shape[0]), 0, _ptr(nu),
                      x0.ctypes.data, _ptr(lam_out), _ptr(A_out), o)
        t = ctypes.c_uint64()
        st = lib().stmf_submit(self.handle, ctypes.byref(req), ctypes.byref(t))
        if st != 0:
            raise StmfError(st, "stmf_submit")
        self._keep[t.value] = (keep, nu, lam_out, A_out)
        return t.value

    def poll(self, ticket, timeout_ms=-1):
        res = RequestResult()
        st = lib().stmf_poll(self.handle, ctypes.c_uint64(ticket), ctypes.byref(res),
                             int(timeout_ms))
        if st == 6:
            return None
        if st != 0:
            raise StmfError(st, "stmf_poll")
        self._keep.pop(ticket, None)
        b = res.best
        return dict(state=res.state, best_start=res.best_start, f=b.f, alpha=b.alpha,
                    g_inf=b.g_inf, iters=b.iters, evals=b.evals, stop=b.stop_reason,
                    status=b.status, total_evals=res.total_evals, t_submit=res.t_submit,
                    t_admit=res.t_admit, t_done=res.t_done, footprint=res.footprint)

    def cancel(self, ticket):
        st = lib().stmf_cancel(self.handle, ctypes.c_uint64(ticket))
        if st != 0:
            raise StmfError(st, "stmf_cancel")

    def stats(self):
        s = ServerStats()
        lib().stmf_server_get_stats(self.handle, ctypes.byref(s))
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().stmf_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class AdamOpts(ctypes.Structure):
    _fields_ = [("lr0", ctypes.c_double), ("lr1", ctypes.c_double), ("beta1", ctypes.c_double),
                ("beta2", ctypes.c_double), ("eps", ctypes.c_double), ("epoch", ctypes.c_int64),
                ("max_epochs", ctypes.c_int64)]


class AdamResult(ctypes.Structure):
    _fields_ = [("f_est", ctypes.c_double), ("epochs", ctypes.c_int64), ("iters", ctypes.c_int64),
                ("drops", ctypes.c_int32), ("status", ctypes.c_int32)]


def _declare_stochastic(L):
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    L.stmf_fg_sampled.argtypes = [vp, ctypes.POINTER(Samples), vp, i64, i32, i64, vp, vp, vp, vp,
                                  vp, vp, vp]
    L.stmf_adam_default_opts.argtypes = [ctypes.POINTER(AdamOpts)]
    L.stmf_adam.argtypes = [vp, ctypes.POINTER(Samples), i32, i64, ctypes.POINTER(AdamOpts), vp,
                            i64, i64, vp, i64, vp, vp, ctypes.POINTER(AdamResult), vp]
    for name in ("stmf_fg_sampled", "stmf_adam_default_opts", "stmf_adam"):
        getattr(L, name).restype = ctypes.c_int


_extra_declarers.append(_declare_stochastic)


def _check_idx(idx, name):
    if idx.dtype != torch.int64 or not idx.is_cuda or not idx.is_contiguous():
        raise ValueError("%s must be a contiguous CUDA int64 tensor" % name)


def fg_sampled(V, idx, d, lam, A, alpha=None, stream=None, ctx=None):
    """stmf_fg_sampled: Alg. 2 on the rows idx of V with weights 1/len(idx) (Lemma 5.1)."""
    ctx = ctx or default_context()
    desc, keep = as_samples(V)
    _check_idx(idx, "idx")
    n, r = desc.n, lam.shape[0]
    f = torch.empty(1, dtype=torch.float64, device=lam.device)
    gl = torch.empty(r, dtype=torch.float64, device=lam.device)
    GA = torch.empty((r, n), dtype=torch.float64, device=lam.device).T
    st = lib().stmf_fg_sampled(ctx.handle, ctypes.byref(desc), _ptr(idx), int(idx.numel()),
                               int(d), int(r), _ptr(lam), _ptr(A), _ptr(alpha), _ptr(f),
                               _ptr(gl), _ptr(GA), _stream(stream))
    ctx.check(st, "stmf_fg_sampled")
    del keep
    return f, gl, GA


def adam(V, d, lam, A, sample_idx, est_idx, stream=None, ctx=None, **kw):
    """stmf_adam: Sec. 5's Adam schedule; sample_idx (iters, s) and est_idx (e,) CUDA int64.
    lam, A (column-major) are updated in place. Returns a dict."""
    ctx = ctx or default_context()
    desc, keep = as_samples(V)
    _check_idx(sample_idx, "sample_idx")
    _check_idx(est_idx, "est_idx")
    o = AdamOpts()
    lib().stmf_adam_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    res = AdamResult()
    iters, s = sample_idx.shape
    st = lib().stmf_adam(ctx.handle, ctypes.byref(desc), int(d), int(lam.shape[0]),
                         ctypes.byref(o), _ptr(sample_idx), int(iters), int(s), _ptr(est_idx),
                         int(est_idx.numel()), _ptr(lam), _ptr(A), ctypes.byref(res),
                         _stream(stream))
    ctx.check(st, "stmf_adam")
    del keep
    return dict(f_est=res.f_est, epochs=res.epochs, iters=res.iters, drops=res.drops,
                status=res.status)


def _declare_rrf(L):
    L.stmf_rrf_start.argtypes = [ctypes.c_void_p, ctypes.POINTER(Samples), ctypes.c_int64,
                                 ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
    L.stmf_rrf_start.restype = ctypes.c_int


_extra_declarers.append(_declare_rrf)


def rrf_start(V, r_hat, seed, stream=None, ctx=None):
    """stmf_rrf_start: A0 = V Omega with unit-norm columns (eq. rrf), Omega drawn on the device
    from Philox4x32-10. Returns A0 as an (n, r_hat) column-major CUDA float64 view."""
    ctx = ctx or default_context()
    desc, keep = as_samples(V)
    A0 = torch.empty((int(r_hat), desc.n), dtype=torch.float64,
                     device=torch.device("cuda", ctx.device)).T
    st = lib().stmf_rrf_start(ctx.handle, ctypes.byref(desc), int(r_hat), ctypes.c_uint64(seed),
                              _ptr(A0), _stream(stream))
    ctx.check(st, "stmf_rrf_start")
    del keep
    return A0


def _declare_sharded(L):
    vp = ctypes.c_void_p
    L.stmf_fg_partial.argtypes = [vp, ctypes.POINTER(Samples), vp, ctypes.c_int64, ctypes.c_int32,
                                  ctypes.c_int64, vp, vp, vp, vp]
    L.stmf_fg_finish.argtypes = [vp, vp, ctypes.c_int64, ctypes.c_int32, ctypes.c_int64, vp, vp,
                                 vp, vp, vp, vp, vp]
    L.stmf_fg_partial.restype = ctypes.c_int
    L.stmf_fg_finish.restype = ctypes.c_int


_extra_declarers.append(_declare_sharded)


def fg_partial(V, nu, p_total, d, lam, A, stream=None, ctx=None):
    """stmf_fg_partial: this shard's [w; vec(Y)] as an (r + n r,) CUDA float64 tensor."""
    ctx = ctx or default_context()
    desc, keep = as_samples(V)
    r = lam.shape[0]
    yw = torch.empty(r + desc.n * r, dtype=torch.float64, device=lam.device)
    st = lib().stmf_fg_partial(ctx.handle, ctypes.byref(desc), _ptr(nu), int(p_total), int(d),
                               int(r), _ptr(lam), _ptr(A), _ptr(yw), _stream(stream))
    ctx.check(st, "stmf_fg_partial")
    del keep
    return yw


def fg_finish(yw, n, d, lam, A, alpha=None, stream=None, ctx=None):
    """stmf_fg_finish: f, g_lambda, G_A from a summed [w; vec(Y)]."""
    ctx = ctx or default_context()
    r = lam.shape[0]
    f = torch.empty(1, dtype=torch.float64, device=lam.device)
    gl = torch.empty(r, dtype=torch.float64, device=lam.device)
    GA = torch.empty((r, n), dtype=torch.float64, device=lam.device).T
    st = lib().stmf_fg_finish(ctx.handle, _ptr(yw), int(n), int(d), int(r), _ptr(lam), _ptr(A),
                              _ptr(alpha), _ptr(f), _ptr(gl), _ptr(GA), _stream(stream))
    ctx.check(st, "stmf_fg_finish")
    return f, gl, GA


def _declare_host(L):
    vp = ctypes.c_void_p
    L.stmf_fg_host.argtypes = [vp, ctypes.POINTER(Samples), vp, ctypes.c_int32, ctypes.c_int64,
                               vp, vp, ctypes.c_double, vp, vp, vp, vp]
    L.stmf_fg_host.restype = ctypes.c_int


_extra_declarers.append(_declare_host)


def fg_host(V, nu, d, lam, A, alpha=0.0, stream=None, ctx=None):
    """stmf_fg_host: the evaluation with host inputs and outputs. V: torch CPU tensor p x ld of a
    storage dtype (pin it for overlapped copies), or a storage dict with CPU tensors; lam (r,) and
    A (n, r) float64 CPU/NumPy. Returns host NumPy (f, g_lambda, G_A)."""
    import numpy as np
    ctx = ctx or default_context()
    scale = None
    n = None
    if isinstance(V, dict):
        n, scale, V = V["n"], V.get("scale"), V["data"]
    if V.is_cuda:
        raise ValueError("fg_host takes samples in host memory")
    dt = _TORCH_DTYPE[V.dtype]
    n = V.shape[1] if n is None else n
    desc = Samples(V.data_ptr(), scale.data_ptr() if scale is not None else None, int(n),
                   int(V.shape[0]), int(V.stride(0)), dt, 0)
    lam_h = np.ascontiguousarray(np.asarray(lam, dtype=np.float64))
    A_h = np.asfortranarray(np.asarray(A, dtype=np.float64))
    nu_h = None if nu is None else np.ascontiguousarray(np.asarray(nu, dtype=np.float64))
    r = lam_h.shape[0]
    f = np.empty(1)
    gl = np.empty(r)
    GA = np.empty((n, r), order="F")
    st = lib().stmf_fg_host(ctx.handle, ctypes.byref(desc),
                            None if nu_h is None else nu_h.ctypes.data, int(d), int(r),
                            lam_h.ctypes.data, A_h.ctypes.data, float(alpha), f.ctypes.data,
                            gl.ctypes.data, GA.ctypes.data, _stream(stream))
    ctx.check(st, "stmf_fg_host")
    return float(f[0]), gl, GA
