"""Parity at the full workload sizes (N = 128^3 = 2,097,152) in the configurations the
benchmark runs.

Two references, both from the CPU oracle:
  * its row-sampled HTLR (Algorithms 1-2 on every block whose target box holds a sampled
    row) on 64 rows chosen to reach every path of the kernels: leaf boxes on every face,
    edge and corner of the leaf grid and in the interior, both parities per dimension
    (the grouped tensor-core kernel works per parity class and zero-fills sources that
    fall outside the domain), and random rows;
  * the FP64 direct sums of the Nystrom product (eq. (1.3)-(1.4)) on 1024 seeded random
    rows, the paper's error measure on sampled rows (§5).
"""
import numpy as np
import pytest

from _helpers import rel

pytestmark = pytest.mark.gpu

TOL = 1e-12        # FP64 and df64 modes against the oracle's HTLR
MIXED_TOL = 1e-6   # FP32 far field, BF16X6 tensor cores: against the oracle's HTLR


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _lines_per_box(coords, nb1):
    """First grid line and count of every 1-D box of a level (half-open cells)."""
    first, cnt = [], []
    for k in range(nb1):
        lo, hi = k / nb1, (k + 1) / nb1
        idx = np.nonzero((coords >= lo) & ((coords < hi) | ((hi >= 1.0) & (coords <= 1.0))))[0]
        first.append(int(idx[0]))
        cnt.append(len(idx))
    return first, cnt


def structured_rows(w, count=64, seed=77):
    """Rows covering every boundary class (low face, interior, high face per dimension:
    27 classes in 3D) of the leaf grid, each class twice with different parities (all 8
    parity classes occur), the rest random; inside a leaf the row alternates between its
    corners, its centre and a random point."""
    nb1 = w.n // w.leaf
    rng = np.random.default_rng(seed)
    coords = w.coords()
    boxes = [_lines_per_box(coords[l], nb1) for l in range(w.d)]
    # per dimension: on the low face, in the interior, on the high face; the first round
    # takes the face boxes themselves, the second the boxes next to them (the other
    # parity); interior boxes alternate parity with the class index
    leaves = []
    for rep in range(2):
        for c in range(3 ** w.d):
            b = []
            for l in range(w.d):
                cls = (c // 3 ** l) % 3
                if cls == 0:
                    b.append(rep)
                elif cls == 2:
                    b.append(nb1 - 1 - rep)
                else:
                    b.append(nb1 // 2 - 1 + ((c + rep + l) & 1))
            leaves.append(b)
    while len(leaves) < count:
        leaves.append([int(v) for v in rng.integers(0, nb1, size=w.d)])
    rows = []
    for i, b in enumerate(leaves[:count]):
        pt = 0
        for l in range(w.d):
            f, c = boxes[l][0][b[l]], boxes[l][1][b[l]]
            mode = i % 4
            j = 0 if mode == 0 else c - 1 if mode == 1 else c // 2 if mode == 2 else int(rng.integers(0, c))
            pt += (f + j) * w.n ** l
        rows.append(pt)
    rows = np.array(sorted(set(rows)), dtype=np.int64)
    return rows


def _run(w, u, grid=None, **kw):
    import torch
    from paper_2508_05958_gb300 import htlr
    H = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, kscale=w.kscale,
                            kparam=w.kparam, a=w.a(), grid=grid, **kw)
    try:
        ud = torch.from_numpy(np.ascontiguousarray(u.T)).cuda()
        fd = torch.empty_like(ud)
        htlr.htlr_matvec(H, ud, fd, u.shape[1])
        htlr.htlr_sync(H)
        return fd.cpu().numpy().T.copy(), htlr.htlr_info(H)
    finally:
        htlr.htlr_free(H)


class _Case:
    """Inputs and oracle references of one full-size workload (computed once)."""

    def __init__(self, oracle, name, nrhs, dense_rows=1024):
        from paper_2508_05958_gb300.workloads import workload
        self.w = w = workload(name)
        self.grid = w.grid()
        self.u = w.u(nrhs=nrhs)
        self.rows = structured_rows(w)
        okw = {} if self.grid is None else {"grid": self.grid, "orth": False}
        self.ref = oracle.htlr_rows(w.d, w.n, w.ktype, w.leaf, w.p, w.eta, self.u, self.rows,
                                    scale=w.kscale, param=w.kparam, a=w.a(), **okw)
        self.drows = w.sample_rows(dense_rows, seed=1024)
        self.dense = oracle.dense_rows(w.d, w.n, w.ktype, self.u, self.drows, scale=w.kscale,
                                       param=w.kparam, grid=self.grid, a=w.a(), q=w.q)

    def check(self, tol_htlr, tol_dense, **kw):
        f, info = _run(self.w, self.u, grid=self.grid, **kw)
        e_h = rel(f[self.rows], self.ref)
        e_d = rel(f[self.drows], self.dense)
        print(f"\n{self.w.name} {kw}: vs oracle HTLR ({len(self.rows)} rows) {e_h:.3e}, "
              f"vs direct sums ({len(self.drows)} rows) {e_d:.3e}")
        assert e_h < tol_htlr, e_h
        assert e_d < tol_dense, e_d
        return info


@pytest.fixture(scope="module")
def c3(oracle):
    return _Case(oracle, "c3", 64)


@pytest.fixture(scope="module")
def c4(oracle):
    return _Case(oracle, "c4", 16)


def test_structured_rows_cover_every_class():
    from paper_2508_05958_gb300.workloads import workload
    for name in ("c3", "c4"):
        w = workload(name)
        rows = structured_rows(w)
        nb1 = w.n // w.leaf
        boxes = [_lines_per_box(w.coords()[l], nb1) for l in range(w.d)]
        seen_bnd, seen_par = set(), set()
        for r in rows:
            idx = [(r // w.n ** l) % w.n for l in range(w.d)]
            b = [max(k for k in range(nb1) if boxes[l][0][k] <= idx[l]) for l in range(w.d)]
            seen_bnd.add(tuple(0 if k <= 1 else 2 if k >= nb1 - 2 else 1 for k in b))
            seen_par.add(tuple(k % 2 for k in b))
        assert len(rows) >= 60
        assert len(seen_bnd) == 27 and len(seen_par) == 8


# Interpolation error of the HTLR product against the direct sums at these settings (Thm
# 3.2: geometric in p), measured with the FP64 path: 3.9e-7 (c3: 1/r, p = 6) and 9e-9
# (c4: exp(-r), p = 7).  Bounds: those values with margin.
C3_INTERP = 1e-6
C4_INTERP = 5e-8


def test_c3_df64(c3):
    info = c3.check(TOL, C3_INTERP, storage=2, far_precision=1, near_precision=1)
    assert info["far_per_level"] == [0, 0, 1416, 133944, 2021592]
    assert info["near_blocks"] == 383272


def test_c3_tensor_cores(c3):
    """The bench's c3 mode: 64 RHS, BF16X6 far and near on the grouped kernel."""
    info = c3.check(MIXED_TOL, C3_INTERP + MIXED_TOL, storage=2, far_precision=3,
                    near_precision=3)
    assert info["tc_grouped"] == (1 << 2) | (1 << 3) | (1 << 4) | -(1 << 31)


@pytest.mark.parametrize("far", [2, 3])
def test_c3_mixed_far_df64_near(c3, far):
    """FP32 or BF16X6 far field with a df64 near field on the CUDA cores."""
    c3.check(MIXED_TOL, C3_INTERP + MIXED_TOL, storage=2, far_precision=far, near_precision=1)


def test_c4_fp64(c4):
    info = c4.check(TOL, C4_INTERP, far_precision=1, near_precision=0)
    assert info["storage"] == 3


def test_c4_tensor_core_far_fp32_near(c4):
    """The bench's c4 mode: 16 RHS, BF16X6 far field (grouped kernel on the tensor grid's
    shared cores), FP32 generated near field."""
    info = c4.check(MIXED_TOL, C4_INTERP + MIXED_TOL, far_precision=3, near_precision=2)
    assert info["storage"] == 3 and info["tc_grouped"] == (1 << 2) | (1 << 3) | (1 << 4)


def test_c4_tensor_cores_far_and_near(c4):
    """The bench's c4 mode: BF16X6 far field on the grouped kernel, the generated near
    field on the tensor cores (TF32X3)."""
    info = c4.check(MIXED_TOL, C4_INTERP + MIXED_TOL, far_precision=3, near_precision=4)
    assert info["storage"] == 3 and info["near_precision"] == 4


def test_c4_tensor_core_far_fp64_near(c4):
    c4.check(MIXED_TOL, C4_INTERP + MIXED_TOL, far_precision=3, near_precision=0)
