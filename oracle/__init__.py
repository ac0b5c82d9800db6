"""CPU oracle for the HTLR construction and matrix-vector product (arXiv 2508.05958).

TEST INFRASTRUCTURE ONLY.  This package wraps ``htlr_oracle.c``, a plain FP64 C
implementation of the Nystrom operator (eq. (1.3)/(1.4)), Construct (Algorithm 1) and
HMultVec (Algorithm 2).  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it; the CUDA
library never does, and the two share no code.

Functions whose result no independent pin covers would say "parity unpinned" here;
every function below is pinned by a test under ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "htlr_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

# Kernel identifiers (interface numbering shared with the library's public enum).
K_LOG, K_INV_R, K_EXP_R, K_GAUSS, K_POLY, K_CONST = range(6)

_D = ctypes.POINTER(ctypes.c_double)
_I64 = ctypes.POINTER(ctypes.c_int64)
_I32 = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, OpenMP)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.orc_kernel_eval.restype = ctypes.c_double
            L.orc_kernel_eval.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_int, _D, _D]
            L.orc_gauss_legendre.restype = ctypes.c_int
            L.orc_gauss_legendre.argtypes = [ctypes.c_int, _D, _D]
            L.orc_diag_integral_eval.restype = ctypes.c_double
            L.orc_diag_integral_eval.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                                 ctypes.c_int, ctypes.c_int, _D, _D, _D]
            L.orc_cheb_nodes.restype = None
            L.orc_cheb_nodes.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, _D]
            L.orc_lagrange.restype = ctypes.c_double
            L.orc_lagrange.argtypes = [ctypes.c_int, _D, ctypes.c_int, ctypes.c_double]
            L.orc_qr.restype = None
            L.orc_qr.argtypes = [ctypes.c_int, ctypes.c_int, _D, _D, _D]
            L.orc_htlr_count.restype = ctypes.c_int
            L.orc_htlr_count.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double, _I64, _I64, _D]
            L.orc_htlr_construct.restype = ctypes.c_void_p
            L.orc_htlr_construct.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_double, _D, _D, _D,
                                             ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                             ctypes.c_int, ctypes.c_int]
            L.orc_htlr_free.restype = None
            L.orc_htlr_free.argtypes = [ctypes.c_void_p]
            L.orc_htlr_stats.restype = ctypes.c_int
            L.orc_htlr_stats.argtypes = [ctypes.c_void_p, _I64, _I64, _D]
            L.orc_htlr_matvec.restype = ctypes.c_int
            L.orc_htlr_matvec.argtypes = [ctypes.c_void_p, _D, ctypes.c_int, _D]
            L.orc_htlr_rows.restype = ctypes.c_int
            L.orc_htlr_rows.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, _D, _D, _D, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_int, _D,
                                        ctypes.c_int, _I64, ctypes.c_int64, _D]
            L.orc_dense_rows_api.restype = ctypes.c_int
            L.orc_dense_rows_api.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_double, _D, _D, _D,
                                             ctypes.c_int, _D, ctypes.c_int, _I64,
                                             ctypes.c_int64, _D]
            L.orc_far_block.restype = ctypes.c_int
            L.orc_far_block.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, _D, _D, ctypes.c_int, _I32, _I32,
                                        ctypes.c_int, ctypes.c_double, ctypes.c_int, _I32, _I32,
                                        _D, _D, _D]
            L.orc_htlr_matvec_range.restype = ctypes.c_double
            L.orc_htlr_matvec_range.argtypes = [ctypes.c_void_p, _D, _D, ctypes.c_long,
                                                ctypes.c_long]
            L.orc_htlr_nblocks.restype = ctypes.c_long
            L.orc_htlr_nblocks.argtypes = [ctypes.c_void_p]
            L.orc_num_threads.restype = ctypes.c_int
            L.orc_num_threads.argtypes = []
            L.orc_set_num_threads.restype = ctypes.c_int
            L.orc_set_num_threads.argtypes = [ctypes.c_int]
            _lib = L
    return _lib


def _dp(a):
    if a is None:
        return None
    return a.ctypes.data_as(_D)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def _grid_arrays(grid, d, n):
    """``grid`` is None (uniform grid of Example 2.1) or a pair (x, edges) with shapes
    (d, n) and (d, n+1)."""
    if grid is None:
        return None, None
    x, e = grid
    x = _f64(np.asarray(x).reshape(d, n))
    e = _f64(np.asarray(e).reshape(d, n + 1))
    return x, e


# ----------------------------------------------------------------------------------
# Elementary pieces
# ----------------------------------------------------------------------------------
def kernel(ktype, x, y, scale=1.0, param=0.0):
    x = _f64(x)
    y = _f64(y)
    return lib().orc_kernel_eval(ktype, scale, param, len(x), _dp(x), _dp(y))


def gauss_legendre(q):
    x = np.zeros(q)
    w = np.zeros(q)
    if lib().orc_gauss_legendre(q, _dp(x), _dp(w)) != 0:
        raise ValueError("q must be >= 1")
    return x, w


def diag_integral(ktype, xi, lo, hi, q=16, scale=1.0, param=0.0):
    """int over the box [lo, hi] of k(xi, y) dy by the subdivided Gauss-Legendre rule."""
    xi, lo, hi = _f64(xi), _f64(lo), _f64(hi)
    return lib().orc_diag_integral_eval(ktype, scale, param, len(xi), q, _dp(xi), _dp(lo),
                                        _dp(hi))


def cheb_nodes(p, a, b):
    xi = np.zeros(p)
    lib().orc_cheb_nodes(p, a, b, _dp(xi))
    return xi


def lagrange(xi, t, x):
    xi = _f64(xi)
    return lib().orc_lagrange(len(xi), _dp(xi), t, float(x))


def qr(A):
    A = np.asfortranarray(A, dtype=np.float64)
    m, c = A.shape
    k = min(m, c)
    Q = np.zeros((m, k), order="F")
    R = np.zeros((k, c), order="F")
    lib().orc_qr(m, c, A.ctypes.data_as(_D), Q.ctypes.data_as(_D), R.ctypes.data_as(_D))
    return Q, R


def num_threads():
    return lib().orc_num_threads()


def set_num_threads(n):
    """Threads of the oracle's OpenMP loops (n <= 0 keeps the current count); returns the
    count in effect."""
    return lib().orc_set_num_threads(int(n))


# ----------------------------------------------------------------------------------
# Block-tree structure
# ----------------------------------------------------------------------------------
def htlr_count(d, n, leaf, p, eta):
    """Counts of the block cluster tree on the uniform grid (Def. 2.4).
    Returns (far_per_level list, near, storage in doubles of the paper's layout)."""
    far = np.zeros(40, dtype=np.int64)
    near = np.zeros(1, dtype=np.int64)
    st = np.zeros(1)
    L = lib().orc_htlr_count(d, n, leaf, p, eta, far.ctypes.data_as(_I64),
                             near.ctypes.data_as(_I64), _dp(st))
    if L < 0:
        raise ValueError("n must be leaf * 2^L")
    return [int(v) for v in far[:L + 1]], int(near[0]), float(st[0])


# ----------------------------------------------------------------------------------
# Dense Nystrom product
# ----------------------------------------------------------------------------------
def dense_rows(d, n, ktype, u, rows=None, scale=1.0, param=0.0, grid=None, a=None, q=16):
    """Rows of f = A u for the Nystrom operator (eq. (1.3), (1.4)); u is N or N x nrhs
    (column-major semantics).  rows=None computes every row."""
    N = n ** d
    u = np.asarray(u, dtype=np.float64)
    vec = u.ndim == 1
    U = np.asfortranarray(u.reshape(N, -1))
    nrhs = U.shape[1]
    rows = np.arange(N, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, np.int64)
    out = np.zeros((len(rows), nrhs), order="F")
    x, e = _grid_arrays(grid, d, n)
    a = _f64(a)
    rc = lib().orc_dense_rows_api(d, n, ktype, scale, param, _dp(x), _dp(e), _dp(a), q,
                                  U.ctypes.data_as(_D), nrhs, rows.ctypes.data_as(_I64),
                                  len(rows), out.ctypes.data_as(_D))
    if rc != 0:
        raise ValueError("invalid dense product arguments")
    return out[:, 0] if vec else out


# ----------------------------------------------------------------------------------
# HTLR: Construct (Algorithm 1) and HMultVec (Algorithm 2)
# ----------------------------------------------------------------------------------
class HTLR:
    """A constructed HTLR matrix held by the oracle (every block stored, paper layout)."""

    def __init__(self, d, n, ktype, leaf, p, eta, scale=1.0, param=0.0, grid=None, a=None,
                 orth=True, q=16):
        self.d, self.n, self.N = d, n, n ** d
        x, e = _grid_arrays(grid, d, n)
        a = _f64(a)
        h = lib().orc_htlr_construct(d, n, ktype, scale, param, _dp(x), _dp(e), _dp(a), leaf,
                                     p, eta, 1 if orth else 0, q)
        if not h:
            raise ValueError("invalid HTLR arguments")
        self._h = h

    def matvec(self, u):
        u = np.asarray(u, dtype=np.float64)
        vec = u.ndim == 1
        U = np.asfortranarray(u.reshape(self.N, -1))
        F = np.zeros_like(U, order="F")
        lib().orc_htlr_matvec(self._h, U.ctypes.data_as(_D), U.shape[1], F.ctypes.data_as(_D))
        return F[:, 0] if vec else F

    def nblocks(self):
        return lib().orc_htlr_nblocks(self._h)

    def matvec_range(self, u, f, k0, k1):
        """Accumulate blocks k0..k1-1 (recursion order) of A u into f (one RHS, both
        float64 arrays of length N); returns the multiply-adds of those blocks."""
        assert u.dtype == np.float64 and f.dtype == np.float64 and u.size == f.size == self.N
        return lib().orc_htlr_matvec_range(self._h, u.ctypes.data_as(_D), f.ctypes.data_as(_D),
                                           k0, k1)

    def stats(self):
        far = np.zeros(40, dtype=np.int64)
        near = np.zeros(1, dtype=np.int64)
        st = np.zeros(1)
        L = lib().orc_htlr_stats(self._h, far.ctypes.data_as(_I64), near.ctypes.data_as(_I64),
                                 _dp(st))
        return [int(v) for v in far[:L + 1]], int(near[0]), float(st[0])

    def free(self):
        if self._h:
            lib().orc_htlr_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def htlr_rows(d, n, ktype, leaf, p, eta, u, rows, scale=1.0, param=0.0, grid=None, a=None,
              orth=True, q=16):
    """Rows of the HTLR product for grids too large to store (blocks built on demand)."""
    N = n ** d
    u = np.asarray(u, dtype=np.float64)
    vec = u.ndim == 1
    U = np.asfortranarray(u.reshape(N, -1))
    rows = np.ascontiguousarray(rows, np.int64)
    out = np.zeros((len(rows), U.shape[1]), order="F")
    x, e = _grid_arrays(grid, d, n)
    a = _f64(a)
    rc = lib().orc_htlr_rows(d, n, ktype, scale, param, _dp(x), _dp(e), _dp(a), leaf, p, eta,
                             1 if orth else 0, q, U.ctypes.data_as(_D), U.shape[1],
                             rows.ctypes.data_as(_I64), len(rows), out.ctypes.data_as(_D))
    if rc != 0:
        raise ValueError("invalid HTLR arguments")
    return out[:, 0] if vec else out


def far_block(d, n, ktype, level, bt, bs, p, eta, scale=1.0, param=0.0, grid=None, orth=True):
    """Factors and core of one admissible block (Algorithm 1).  Returns None when the
    pair is not admissible, else (U list, V list, G matrix prod(pt) x prod(ps))."""
    x, e = _grid_arrays(grid, d, n)
    nb = n >> level
    maxcnt = n  # generous for tensor grids
    U = np.zeros(d * maxcnt * p)
    V = np.zeros(d * maxcnt * p)
    G = np.zeros(p ** (2 * d))
    pt = np.zeros(3, dtype=np.int32)
    ps = np.zeros(3, dtype=np.int32)
    bt = np.ascontiguousarray(list(bt) + [0] * (3 - d), np.int32)
    bs = np.ascontiguousarray(list(bs) + [0] * (3 - d), np.int32)
    rc = lib().orc_far_block(d, n, ktype, scale, param, _dp(x), _dp(e), level,
                             bt.ctypes.data_as(_I32), bs.ctypes.data_as(_I32), p, eta,
                             1 if orth else 0, pt.ctypes.data_as(_I32),
                             ps.ctypes.data_as(_I32), _dp(U), _dp(V), _dp(G))
    if rc < 0:
        raise ValueError("bad arguments")
    if rc == 1:
        return None
    # split the concatenated factors (uniform grid: nb points per dimension)
    Us, Vs, ou, ov = [], [], 0, 0
    cnt_t = [nb] * d if grid is None else None
    if cnt_t is None:
        raise NotImplementedError("far_block factors are split for uniform grids only")
    for l in range(d):
        Us.append(U[ou:ou + nb * pt[l]].reshape(pt[l], nb).T.copy())
        Vs.append(V[ov:ov + nb * ps[l]].reshape(ps[l], nb).T.copy())
        ou += nb * pt[l]
        ov += nb * ps[l]
    nt = int(np.prod(pt[:d]))
    ns = int(np.prod(ps[:d]))
    Gm = G[:nt * ns].reshape(ns, nt).T.copy()
    return Us, Vs, Gm
