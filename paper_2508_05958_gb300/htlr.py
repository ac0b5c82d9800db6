"""Python binding of the HTLR C ABI (include/htlr.h): argument marshalling only.

Every call goes to ``libhtlr.so`` (hand-written sm_103a CUDA); there is no Python or
CPU fallback.  Device buffers are PyTorch CUDA tensors (or raw device pointers).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

HTLR_OK, HTLR_EINVAL, HTLR_ENOMEM, HTLR_ECUDA, HTLR_EUNSUPPORTED, HTLR_ETIMEOUT, HTLR_EDEVICE = (
    0, -1, -2, -3, -4, -5, -6)
K_LOG, K_INV_R, K_EXP_R, K_GAUSS, K_POLY, K_CONST = range(6)
GRID_UNIFORM, GRID_TENSOR = 0, 1
STORE_AUTO, STORE_STORED, STORE_SHARED = 0, 1, 2
PREC_FP64, PREC_DF64, PREC_FP32, PREC_BF16X6, PREC_TF32X3 = 0, 1, 2, 3, 4
MAX_LEVELS = 16

NUM_STAGES = 5
SYMBOLS = ("htlr_construct", "htlr_construct_ex", "htlr_matvec", "htlr_matvec_timed",
           "htlr_matvec_host", "htlr_matvec_noalloc", "htlr_gmres", "htlr_free",
           "htlr_info", "htlr_set_stream", "htlr_sync", "htlr_last_error",
           "htlr_last_launch_count", "htlr_plan_create", "htlr_plan_launch",
           "htlr_plan_launches", "htlr_plan_free", "htlr_autotune", "htlr_autotune_clear_cache",
           "htlr_server_create", "htlr_server_add_operator", "htlr_server_submit",
           "htlr_server_poll", "htlr_server_wait", "htlr_server_get_stats",
           "htlr_server_destroy", "htlr_tensor_flops", "htlr_set_wait_limit",
           "htlr_device_allocations")


class HTLRError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"HTLR error {code}: {msg}")
        self.code = code


class htlr_kernel(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("scale", ctypes.c_double), ("param", ctypes.c_double)]


class htlr_grid(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int), ("coords", ctypes.POINTER(ctypes.c_double)),
                ("edges", ctypes.POINTER(ctypes.c_double)), ("a", ctypes.POINTER(ctypes.c_double))]


class htlr_options(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int), ("orth", ctypes.c_int), ("quad_order", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("hbm_limit", ctypes.c_size_t),
                ("far_precision", ctypes.c_int), ("near_precision", ctypes.c_int),
                ("tc_segment", ctypes.c_int), ("tc_flush", ctypes.c_int),
                ("tc_wait_cycles", ctypes.c_longlong)]


class htlr_stats(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", ctypes.c_int), ("levels", ctypes.c_int),
                ("p", ctypes.c_int), ("p_eff_leaf", ctypes.c_int), ("storage", ctypes.c_int),
                ("far_per_level", ctypes.c_int64 * MAX_LEVELS), ("near_blocks", ctypes.c_int64),
                ("unique_cores", ctypes.c_int64), ("unique_near", ctypes.c_int64),
                ("paper_storage_doubles", ctypes.c_double), ("bytes_cores", ctypes.c_size_t),
                ("bytes_near", ctypes.c_size_t), ("bytes_factors", ctypes.c_size_t),
                ("bytes_work", ctypes.c_size_t), ("bytes_total", ctypes.c_size_t),
                ("diag_value", ctypes.c_double), ("far_precision", ctypes.c_int),
                ("near_precision", ctypes.c_int), ("tc_grouped", ctypes.c_int),
                ("near_point_pairs", ctypes.c_int64)]


class htlr_gmres_options(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_iters", ctypes.c_int), ("tol", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("max_refine", ctypes.c_int)]


class htlr_gmres_result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("matvecs", ctypes.c_int),
                ("refinements", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("converged", ctypes.c_int)]


class htlr_tune_result(ctypes.Structure):
    _fields_ = [("task_bytes", ctypes.c_size_t), ("stream_ctas_per_sm", ctypes.c_int),
                ("stream_threads", ctypes.c_int), ("tc_stages", ctypes.c_int),
                ("ms", ctypes.c_float), ("default_ms", ctypes.c_float),
                ("candidates", ctypes.c_int), ("from_cache", ctypes.c_int)]


class htlr_server_options(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("max_active", ctypes.c_int),
                ("max_batch", ctypes.c_int), ("mixed", ctypes.c_int),
                ("inner_precision", ctypes.c_int), ("restart", ctypes.c_int),
                ("tol", ctypes.c_double), ("inner_tol", ctypes.c_double),
                ("max_iters", ctypes.c_int), ("use_graphs", ctypes.c_int),
                ("autotune_ms", ctypes.c_double)]


class htlr_operator_spec(ctypes.Structure):
    _fields_ = [("kernel_type", ctypes.c_int), ("kscale", ctypes.c_double),
                ("kparam", ctypes.c_double), ("d", ctypes.c_int), ("n", ctypes.c_int),
                ("leaf", ctypes.c_int), ("r", ctypes.c_int), ("eta", ctypes.c_double),
                ("a", ctypes.POINTER(ctypes.c_double)), ("storage", ctypes.c_int)]


class htlr_request_info(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("error", ctypes.c_int), ("iterations", ctypes.c_int),
                ("matvecs", ctypes.c_int), ("refinements", ctypes.c_int),
                ("rel_residual", ctypes.c_double), ("converged", ctypes.c_int),
                ("submit_s", ctypes.c_double), ("admit_s", ctypes.c_double),
                ("done_s", ctypes.c_double)]


class htlr_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("failed", ctypes.c_longlong), ("active", ctypes.c_int), ("pending", ctypes.c_int),
                ("steps", ctypes.c_longlong), ("batched_matvecs", ctypes.c_longlong),
                ("matvec_columns", ctypes.c_longlong), ("max_batch_seen", ctypes.c_int),
                ("constructions", ctypes.c_longlong), ("evictions", ctypes.c_longlong),
                ("bytes_in_use", ctypes.c_longlong), ("bytes_peak", ctypes.c_longlong),
                ("bytes_budget", ctypes.c_longlong), ("resident_operators", ctypes.c_int)]


REQ_QUEUED, REQ_ACTIVE, REQ_DONE, REQ_FAILED = 0, 1, 2, 3

_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libhtlr.so (building it with nvcc if it is missing).  Raises if neither works:
    the library never falls back to another implementation."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if build_if_missing and (not os.path.exists(path) or _build._stale()):
            _build.build()
        if not os.path.exists(path):
            raise RuntimeError(f"libhtlr.so not found at {path}; run __graft_entry__.build()")
        try:
            import torch  # noqa: F401  (load the CUDA runtime PyTorch uses first)
        except Exception:
            pass
        L = ctypes.CDLL(path)
        P = ctypes.POINTER
        vp = ctypes.c_void_p
        L.htlr_construct.argtypes = [P(vp), P(htlr_kernel), ctypes.c_int, ctypes.c_int,
                                     P(htlr_grid), ctypes.c_int, ctypes.c_int, ctypes.c_double]
        L.htlr_construct.restype = ctypes.c_int
        L.htlr_construct_ex.argtypes = L.htlr_construct.argtypes + [P(htlr_options)]
        L.htlr_construct_ex.restype = ctypes.c_int
        L.htlr_matvec.argtypes = [vp, vp, vp, ctypes.c_int]
        L.htlr_matvec.restype = ctypes.c_int
        L.htlr_matvec_timed.argtypes = [vp, vp, vp, ctypes.c_int, P(ctypes.c_float)]
        L.htlr_matvec_timed.restype = ctypes.c_int
        L.htlr_gmres.argtypes = [vp, vp, vp, vp, ctypes.c_int, P(htlr_gmres_options),
                                 P(htlr_gmres_result)]
        L.htlr_gmres.restype = ctypes.c_int
        L.htlr_matvec_noalloc.argtypes = [vp, vp, vp, ctypes.c_int]
        L.htlr_matvec_noalloc.restype = ctypes.c_int
        L.htlr_matvec_host.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int]
        L.htlr_matvec_host.restype = ctypes.c_int
        L.htlr_free.argtypes = [vp]
        L.htlr_free.restype = None
        L.htlr_info.argtypes = [vp, P(htlr_stats)]
        L.htlr_info.restype = ctypes.c_int
        L.htlr_set_stream.argtypes = [vp, vp]
        L.htlr_set_stream.restype = ctypes.c_int
        L.htlr_sync.argtypes = [vp]
        L.htlr_sync.restype = ctypes.c_int
        L.htlr_device_allocations.argtypes = []
        L.htlr_device_allocations.restype = ctypes.c_longlong
        L.htlr_set_wait_limit.argtypes = [vp, ctypes.c_longlong]
        L.htlr_set_wait_limit.restype = ctypes.c_int
        L.htlr_last_error.argtypes = []
        L.htlr_last_error.restype = ctypes.c_char_p
        L.htlr_last_launch_count.argtypes = [vp]
        L.htlr_last_launch_count.restype = ctypes.c_int
        L.htlr_plan_create.argtypes = [vp, vp, vp, ctypes.c_int, P(vp)]
        L.htlr_plan_create.restype = ctypes.c_int
        L.htlr_plan_launch.argtypes = [vp]
        L.htlr_plan_launch.restype = ctypes.c_int
        L.htlr_plan_launches.argtypes = [vp]
        L.htlr_plan_launches.restype = ctypes.c_int
        L.htlr_plan_free.argtypes = [vp]
        L.htlr_plan_free.restype = None
        L.htlr_autotune.argtypes = [vp, ctypes.c_int, ctypes.c_double, P(htlr_tune_result)]
        L.htlr_autotune.restype = ctypes.c_int
        L.htlr_autotune_clear_cache.argtypes = []
        L.htlr_autotune_clear_cache.restype = None
        L.htlr_tensor_flops.argtypes = [vp, ctypes.c_int]
        L.htlr_tensor_flops.restype = ctypes.c_double
        L.htlr_server_create.argtypes = [P(htlr_server_options), P(vp)]
        L.htlr_server_create.restype = ctypes.c_int
        L.htlr_server_add_operator.argtypes = [vp, P(htlr_operator_spec), P(ctypes.c_int)]
        L.htlr_server_add_operator.restype = ctypes.c_int
        L.htlr_server_submit.argtypes = [vp, ctypes.c_int, P(ctypes.c_double), P(ctypes.c_double),
                                         P(ctypes.c_longlong)]
        L.htlr_server_submit.restype = ctypes.c_int
        L.htlr_server_poll.argtypes = [vp, ctypes.c_longlong, P(htlr_request_info)]
        L.htlr_server_poll.restype = ctypes.c_int
        L.htlr_server_wait.argtypes = [vp, ctypes.c_longlong, ctypes.c_double,
                                       P(htlr_request_info)]
        L.htlr_server_wait.restype = ctypes.c_int
        L.htlr_server_get_stats.argtypes = [vp, P(htlr_server_stats)]
        L.htlr_server_get_stats.restype = ctypes.c_int
        L.htlr_server_destroy.argtypes = [vp]
        L.htlr_server_destroy.restype = None
        _lib = L
        return L


def htlr_last_error() -> str:
    return load().htlr_last_error().decode()


def _check(rc):
    if rc != HTLR_OK:
        raise HTLRError(rc, htlr_last_error())


def _dptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return x.data_ptr()


def _hptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def htlr_construct(ktype, d, n, leaf, r, eta, *, kscale=1.0, kparam=0.0, a=None, grid=None,
                   storage=STORE_AUTO, orth=-1, quad_order=0, stream=None, hbm_limit=0,
                   far_precision=0, near_precision=0, tc_segment=0, tc_flush=0,
                   tc_wait_cycles=0):
    """Construct (Algorithm 1).  ``a``: host array of N values (natural order) or None.
    ``grid``: None (uniform) or (coords (d, n), edges (d, n+1)).  Returns an opaque handle
    (int).  ``stream``: a torch.cuda.Stream, a raw cudaStream_t int, or None."""
    L = load()
    k = htlr_kernel(ktype, kscale, kparam)
    keep = []
    g = htlr_grid()
    g.type = GRID_UNIFORM
    if grid is not None:
        c = np.ascontiguousarray(grid[0], dtype=np.float64)
        e = np.ascontiguousarray(grid[1], dtype=np.float64)
        keep += [c, e]
        g.type = GRID_TENSOR
        g.coords = _hptr(c)
        g.edges = _hptr(e)
    if a is not None:
        a = np.ascontiguousarray(a, dtype=np.float64)
        keep.append(a)
        g.a = _hptr(a)
    o = htlr_options(storage, orth, quad_order, _stream_ptr(stream), hbm_limit, far_precision,
                     near_precision, tc_segment, tc_flush, tc_wait_cycles)
    h = ctypes.c_void_p()
    _check(L.htlr_construct_ex(ctypes.byref(h), ctypes.byref(k), d, n, ctypes.byref(g), leaf, r,
                               eta, ctypes.byref(o)))
    return h.value


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def htlr_matvec(H, u, f, nrhs=None):
    """f = A u with device buffers (torch CUDA tensors, N x nrhs column-major: i.e. a
    contiguous tensor of shape (nrhs, N), or raw pointers with nrhs given)."""
    if nrhs is None:
        nrhs = 1 if u.dim() == 1 else u.shape[0]
    _check(load().htlr_matvec(H, _dptr(u), _dptr(f), nrhs))


def htlr_gmres(H, f, u, nrhs=None, H_inner=None, restart=30, max_iters=3000, tol=1e-10,
               inner_tol=1e-6, max_refine=20) -> dict:
    """Solve A u = f (A = a I + K applied by H) with restarted GMRES; with H_inner, by
    iterative refinement around inner solves with H_inner.  u: initial guess, overwritten.
    Returns the result counters as a dict."""
    if nrhs is None:
        nrhs = 1 if f.dim() == 1 else f.shape[0]
    o = htlr_gmres_options(restart, max_iters, tol, inner_tol, max_refine)
    r = htlr_gmres_result()
    _check(load().htlr_gmres(H, H_inner, _dptr(f), _dptr(u), nrhs, ctypes.byref(o),
                             ctypes.byref(r)))
    return {name: getattr(r, name) for name, _ in htlr_gmres_result._fields_}


def htlr_matvec_noalloc(H, u, f, nrhs=None):
    """f = A u like htlr_matvec, with the library's static 64 MiB scratch instead of any
    device allocation (for callers that cannot allocate; calls on a device share it)."""
    if nrhs is None:
        nrhs = 1 if u.dim() == 1 else u.shape[0]
    _check(load().htlr_matvec_noalloc(H, _dptr(u), _dptr(f), nrhs))


def htlr_matvec_timed(H, u, f, nrhs=None):
    """htlr_matvec that returns the device milliseconds of its stages
    (up, stream, reduce, out), measured with CUDA events on the handle's stream."""
    if nrhs is None:
        nrhs = 1 if u.dim() == 1 else u.shape[0]
    ms = (ctypes.c_float * NUM_STAGES)()
    _check(load().htlr_matvec_timed(H, _dptr(u), _dptr(f), nrhs, ms))
    return list(ms)


def htlr_matvec_host(H, u, f, nrhs):
    """f = A u with host numpy arrays (N * nrhs doubles each, column-major)."""
    assert u.dtype == np.float64 and f.dtype == np.float64
    assert u.flags["F_CONTIGUOUS"] or u.flags["C_CONTIGUOUS"]
    _check(load().htlr_matvec_host(H, _hptr(u), _hptr(f), nrhs))


def htlr_free(H):
    load().htlr_free(H)


def htlr_info(H) -> dict:
    s = htlr_stats()
    _check(load().htlr_info(H, ctypes.byref(s)))
    out = {name: getattr(s, name) for name, _ in htlr_stats._fields_}
    out["far_per_level"] = list(s.far_per_level)[: s.levels + 1]
    return out


def htlr_set_stream(H, stream):
    _check(load().htlr_set_stream(H, _stream_ptr(stream)))


def htlr_sync(H):
    """Wait for the handle's stream; raise HTLRError (code HTLR_ETIMEOUT or HTLR_EDEVICE)
    if a device check failed since the last report (the report clears it)."""
    _check(load().htlr_sync(H))


def htlr_set_wait_limit(H, cycles):
    """Bounded-wait limit of the tensor-core kernels in SM cycles (0: the default)."""
    _check(load().htlr_set_wait_limit(H, int(cycles)))


def htlr_last_launch_count(H) -> int:
    return load().htlr_last_launch_count(H)


class Operator:
    """Convenience owner of a handle: ``op(u)`` returns A u for a CUDA tensor u of shape
    (N,) or (nrhs, N)."""

    def __init__(self, ktype, d, n, leaf, r, eta, **kw):
        self.d, self.n, self.N = d, n, n ** d
        self.handle = htlr_construct(ktype, d, n, leaf, r, eta, **kw)

    def __call__(self, u, out=None):
        import torch
        if out is None:
            out = torch.empty_like(u)
        htlr_matvec(self.handle, u, out)
        return out

    def info(self):
        return htlr_info(self.handle)

    def close(self):
        if self.handle:
            htlr_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def htlr_plan_create(H, u, f, nrhs=None):
    """Capture f = A u (fixed device buffers) into a CUDA graph; returns the plan (int)."""
    if nrhs is None:
        nrhs = 1 if u.dim() == 1 else u.shape[0]
    P = ctypes.c_void_p()
    _check(load().htlr_plan_create(H, _dptr(u), _dptr(f), nrhs, ctypes.byref(P)))
    return P.value


def htlr_plan_launch(P):
    _check(load().htlr_plan_launch(P))


def htlr_plan_launches(P) -> int:
    return load().htlr_plan_launches(P)


def htlr_plan_free(P):
    load().htlr_plan_free(P)


def htlr_autotune(H, nrhs=1, budget_ms=2000.0) -> dict:
    """Time launch-shape candidates for nrhs right-hand sides and apply the fastest."""
    r = htlr_tune_result()
    _check(load().htlr_autotune(H, nrhs, float(budget_ms), ctypes.byref(r)))
    return {k: getattr(r, k) for k, _ in htlr_tune_result._fields_}


def htlr_autotune_clear_cache():
    load().htlr_autotune_clear_cache()


def _struct_dict(x):
    return {k: getattr(x, k) for k, _ in x._fields_}


def server_options(**kw) -> htlr_server_options:
    """Options with the library's defaults (see htlr_server_create) overridden by kw."""
    o = htlr_server_options(0, 64, 16, 1, PREC_FP32, 30, 1e-10, 1e-4, 3000, 1, 0.0)
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Server:
    """Continuous-batching solve server (htlr_server_*): submit(op, f) -> request id,
    wait(id) -> (u, info).  Host numpy arrays in and out."""

    def __init__(self, **options):
        self._L = load()
        self._o = server_options(**options)
        h = ctypes.c_void_p()
        _check(self._L.htlr_server_create(ctypes.byref(self._o), ctypes.byref(h)))
        self._h = h.value
        self._keep = {}      # request id -> output array (must outlive the request)
        self._N = {}

    def add_operator(self, ktype, d, n, leaf, r, eta, *, kscale=1.0, kparam=0.0, a=None,
                     storage=STORE_AUTO) -> int:
        a = None if a is None else np.ascontiguousarray(a, dtype=np.float64)
        spec = htlr_operator_spec(ktype, kscale, kparam, d, n, leaf, r, eta, _hptr(a), storage)
        op = ctypes.c_int()
        _check(self._L.htlr_server_add_operator(self._h, ctypes.byref(spec), ctypes.byref(op)))
        self._N[op.value] = n ** d
        return op.value

    def submit(self, op, f) -> int:
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        if op in self._N and f.size != self._N[op]:
            raise ValueError("f must hold N values")
        u = np.zeros_like(f)
        rid = ctypes.c_longlong()
        _check(self._L.htlr_server_submit(self._h, op, _hptr(f), _hptr(u), ctypes.byref(rid)))
        self._keep[rid.value] = u
        return rid.value

    def poll(self, rid) -> dict:
        info = htlr_request_info()
        _check(self._L.htlr_server_poll(self._h, rid, ctypes.byref(info)))
        return _struct_dict(info)

    def wait(self, rid, timeout_s=-1.0):
        info = htlr_request_info()
        _check(self._L.htlr_server_wait(self._h, rid, float(timeout_s), ctypes.byref(info)))
        return self._keep.pop(rid), _struct_dict(info)

    def stats(self) -> dict:
        st = htlr_server_stats()
        _check(self._L.htlr_server_get_stats(self._h, ctypes.byref(st)))
        return _struct_dict(st)

    def close(self):
        if self._h:
            self._L.htlr_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def htlr_tensor_flops(H, nrhs) -> float:
    """Tensor-core FLOPs one matvec of nrhs right-hand sides executes (0 without BF16X6)."""
    return load().htlr_tensor_flops(H, nrhs)
