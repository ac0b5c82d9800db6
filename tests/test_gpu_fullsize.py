"""Parity at the full workload sizes (N = 128^3 = 2,097,152) in the configuration the
benchmark runs, on outputs the oracle computes row by row (its row-sampled HTLR builds
only the blocks whose target box holds a sampled row)."""
import numpy as np
import pytest

from _helpers import rel

pytestmark = pytest.mark.gpu

TOL = 1e-12
MIXED_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


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


def test_c3_full_size_sampled_rows(oracle):
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c3")
    u = w.u(nrhs=2)
    rows = w.sample_rows(6, seed=11)
    ref = oracle.htlr_rows(w.d, w.n, w.ktype, w.leaf, w.p, w.eta, u, rows, a=w.a())
    f, info = _run(w, u, storage=2, far_precision=1, near_precision=1)
    assert info["far_per_level"] == [0, 0, 1416, 133944, 2021592]
    assert info["near_blocks"] == 383272
    assert rel(f[rows], ref) < TOL
    fm, _ = _run(w, u, storage=2, far_precision=2, near_precision=1)
    assert rel(fm[rows], ref) < MIXED_TOL


def test_c4_full_size_sampled_rows(oracle):
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c4")
    grid = w.grid()
    u = w.u(nrhs=1)
    rows = w.sample_rows(6, seed=12)
    ref = oracle.htlr_rows(w.d, w.n, w.ktype, w.leaf, w.p, w.eta, u, rows, grid=grid,
                           orth=False)
    f, info = _run(w, u, grid=grid, far_precision=1, near_precision=0)
    assert info["storage"] == 3
    assert rel(f[rows], ref) < TOL
    fm, _ = _run(w, u, grid=grid, far_precision=2, near_precision=0)
    assert rel(fm[rows], ref) < MIXED_TOL


TC_TOL = 1e-5     # grouped tensor-core kernel, segmented accumulation (measured 1.8e-6)


def test_c3_full_size_tensor_cores_64_rhs(oracle):
    """c3 as its tensor-core bench variant runs it: 64 RHS, SHARED, BF16X6 far and near
    on the grouped kernel; and the BF16X6 far field with a df64 near field."""
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c3")
    u = w.u(nrhs=64)
    rows = w.sample_rows(4, seed=13)
    ref = oracle.htlr_rows(w.d, w.n, w.ktype, w.leaf, w.p, w.eta, u, rows, a=w.a())
    f, info = _run(w, u, storage=2, far_precision=3, near_precision=3)
    assert info["tc_grouped"] == (1 << 2) | (1 << 3) | (1 << 4) | -(1 << 31)
    assert rel(f[rows], ref) < TC_TOL
    fn, _ = _run(w, u, storage=2, far_precision=3, near_precision=1)
    assert rel(fn[rows], ref) < TC_TOL


def test_c4_full_size_tensor_core_far_fp32_near(oracle):
    """c4 as its bench variant runs it: 16 RHS, BF16X6 far field (grouped kernel on the
    tensor grid's shared cores), FP32 generated near field."""
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c4")
    grid = w.grid()
    u = w.u(nrhs=16)
    rows = w.sample_rows(4, seed=14)
    ref = oracle.htlr_rows(w.d, w.n, w.ktype, w.leaf, w.p, w.eta, u, rows, grid=grid,
                           orth=False)
    f, info = _run(w, u, grid=grid, far_precision=3, near_precision=2)
    assert info["storage"] == 3 and info["tc_grouped"] == (1 << 2) | (1 << 3) | (1 << 4)
    assert rel(f[rows], ref) < TC_TOL
