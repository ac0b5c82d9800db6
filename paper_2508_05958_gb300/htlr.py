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
PREC_FP64, PREC_DF64, PREC_FP32, PREC_BF16X6 = 0, 1, 2, 3
MAX_LEVELS = 16

NUM_STAGES = 4
SYMBOLS = ("htlr_construct", "htlr_construct_ex", "htlr_matvec", "htlr_matvec_timed",
           "htlr_matvec_host", "htlr_matvec_noalloc", "htlr_gmres", "htlr_free",
           "htlr_info", "htlr_set_stream", "htlr_sync", "htlr_last_error",
           "htlr_last_launch_count")


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
                ("far_precision", ctypes.c_int), ("near_precision", ctypes.c_int)]


class htlr_stats(ctypes.Structure):
    _fields_ = [("d", ctypes.c_int), ("n", ctypes.c_int), ("levels", ctypes.c_int),
                ("p", ctypes.c_int), ("p_eff_leaf", ctypes.c_int), ("storage", ctypes.c_int),
                ("far_per_level", ctypes.c_int64 * MAX_LEVELS), ("near_blocks", ctypes.c_int64),
                ("unique_cores", ctypes.c_int64), ("unique_near", ctypes.c_int64),
                ("paper_storage_doubles", ctypes.c_double), ("bytes_cores", ctypes.c_size_t),
                ("bytes_near", ctypes.c_size_t), ("bytes_factors", ctypes.c_size_t),
                ("bytes_work", ctypes.c_size_t), ("bytes_total", ctypes.c_size_t),
                ("diag_value", ctypes.c_double), ("far_precision", ctypes.c_int),
                ("near_precision", ctypes.c_int)]


class htlr_gmres_options(ctypes.Structure):
    _fields_ = [("restart", ctypes.c_int), ("max_iters", ctypes.c_int), ("tol", ctypes.c_double),
                ("inner_tol", ctypes.c_double), ("max_refine", ctypes.c_int)]


class htlr_gmres_result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("matvecs", ctypes.c_int),
                ("refinements", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("converged", ctypes.c_int)]


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
        L.htlr_last_error.argtypes = []
        L.htlr_last_error.restype = ctypes.c_char_p
        L.htlr_last_launch_count.argtypes = [vp]
        L.htlr_last_launch_count.restype = ctypes.c_int
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
                   far_precision=0, near_precision=0):
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
                     near_precision)
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
    _check(load().htlr_sync(H))


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
