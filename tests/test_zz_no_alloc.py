"""htlr_matvec_noalloc: the allocation-free matvec for callers that cannot call
cudaMalloc when they apply an operator (memory fully reserved by a pool or budget,
latency-bound loops that must not block in the allocator, handles shared between
threads).  Its scratch is the library's static 64 MiB device array.

Checked through the C ABI against htlr_matvec, on two calls in a row (the second call
reuses the array the first one left behind).  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    from paper_2508_05958_gb300 import htlr
    return htlr.load()


def _construct(w, storage=1):
    from paper_2508_05958_gb300 import htlr
    return htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, kscale=w.kscale,
                               kparam=w.kparam, a=w.a(), storage=storage)


def _rel(a, b):
    return max(np.linalg.norm(a[c] - b[c]) / np.linalg.norm(b[c]) for c in range(b.shape[0]))


@pytest.mark.parametrize("name,over,nrhs", [("c1", {}, 3), ("c2", {}, 1), ("c2", {"n": 16}, 5)])
def test_noalloc_matches_matvec_twice(lib, name, over, nrhs):
    import torch
    from paper_2508_05958_gb300 import htlr
    from paper_2508_05958_gb300.workloads import workload
    w = workload(name, **over)
    H = _construct(w)
    try:
        u = torch.from_numpy(np.ascontiguousarray(w.u(nrhs=nrhs).T)).cuda()
        ref = torch.empty_like(u)
        assert lib.htlr_matvec(H, u.data_ptr(), ref.data_ptr(), nrhs) == 0
        assert lib.htlr_sync(H) == 0
        refh = ref.cpu().numpy()
        for call in range(2):
            f = torch.full_like(u, float("nan"))
            rc = lib.htlr_matvec_noalloc(H, u.data_ptr(), f.data_ptr(), nrhs)
            assert rc == 0, htlr.htlr_last_error()
            assert lib.htlr_sync(H) == 0
            fh = f.cpu().numpy()
            assert np.all(np.isfinite(fh))
            assert _rel(fh, refh) < TOL, (call, _rel(fh, refh))
    finally:
        htlr.htlr_free(H)


def test_noalloc_makes_no_device_allocation(lib):
    """Every device allocation of the library goes through one counted helper: the count
    does not move across allocation-free calls (an allocation followed by a free inside
    the call would leave free memory unchanged but move the count), and free device
    memory stays the same too."""
    import torch
    from paper_2508_05958_gb300 import htlr
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c1")
    H = _construct(w)
    try:
        u = torch.from_numpy(np.ascontiguousarray(w.u(nrhs=1).T)).cuda()
        f = torch.empty_like(u)
        assert lib.htlr_matvec_noalloc(H, u.data_ptr(), f.data_ptr(), 1) == 0   # first call
        torch.cuda.synchronize()
        n0 = lib.htlr_device_allocations()
        free0 = torch.cuda.mem_get_info()[0]
        for _ in range(3):
            assert lib.htlr_matvec_noalloc(H, u.data_ptr(), f.data_ptr(), 1) == 0
        torch.cuda.synchronize()
        assert lib.htlr_device_allocations() == n0
        assert torch.cuda.mem_get_info()[0] == free0
        # the counter does count: the host-buffer entry point stages its vectors once
        uh = np.ascontiguousarray(w.u(nrhs=1).T)
        fh = np.zeros_like(uh)
        htlr.htlr_matvec_host(H, np.asfortranarray(uh.T), np.asfortranarray(fh.T), 1)
        assert lib.htlr_device_allocations() > n0
    finally:
        htlr.htlr_free(H)


def _paths():
    """Operators that take the other paths of the allocation-free matvec: a generated near
    field on a quasi-uniform tensor grid (on the CUDA cores, and on the tensor cores in
    two passes of 16 RHS), df64 and FP32 block lists, SHARED storage."""
    from paper_2508_05958_gb300.workloads import Workload, quasi_uniform_tensor_grid, workload
    tq = Workload("tq", d=3, n=16, ktype=2, leaf=4, p=4, eta=1.0, seed=41)
    return [
        ("generated near, tensor grid", tq, dict(grid=quasi_uniform_tensor_grid(3, 16, 9)), 3),
        ("df64, STORED", workload("c2", n=16), dict(storage=1, far_precision=1, near_precision=1), 2),
        ("FP32 far / df64 near, SHARED", workload("c2", n=16),
         dict(storage=2, far_precision=2, near_precision=1), 4),
        ("FP64, SHARED", workload("c1"), dict(storage=2), 1),
        ("TF32X3 generated near, tensor grid", tq,
         dict(grid=quasi_uniform_tensor_grid(3, 16, 9), near_precision=4), 17),
    ]


@pytest.mark.parametrize("case", range(5))
def test_noalloc_other_paths_equal_matvec_bitwise(lib, case):
    """The allocation-free matvec runs the same kernels on the same data in the same
    order as htlr_matvec, only with other scratch addresses: the results are equal bit for
    bit, on two calls in a row."""
    import torch
    from paper_2508_05958_gb300 import htlr
    name, w, kw, nrhs = _paths()[case]
    H = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, kscale=w.kscale,
                            kparam=w.kparam, a=w.a(), **kw)
    try:
        u = torch.from_numpy(np.ascontiguousarray(w.u(nrhs=nrhs).T)).cuda()
        ref = torch.empty_like(u)
        assert lib.htlr_matvec(H, u.data_ptr(), ref.data_ptr(), nrhs) == 0
        assert lib.htlr_sync(H) == 0
        for call in range(2):
            f = torch.full_like(u, float("nan"))
            rc = lib.htlr_matvec_noalloc(H, u.data_ptr(), f.data_ptr(), nrhs)
            assert rc == 0, (name, htlr.htlr_last_error())
            assert lib.htlr_sync(H) == 0
            assert torch.equal(f, ref), (name, call)
    finally:
        htlr.htlr_free(H)


def test_noalloc_rejects_operators_above_the_static_maximum(lib):
    import torch
    from paper_2508_05958_gb300 import htlr
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2", n=64)                       # ~0.6 M blocks: scratch well above 64 MiB
    H = _construct(w, storage=2)
    try:
        u = torch.zeros((1, w.N), dtype=torch.float64, device="cuda")
        f = torch.zeros_like(u)
        rc = lib.htlr_matvec_noalloc(H, u.data_ptr(), f.data_ptr(), 1)
        assert rc == htlr.HTLR_ENOMEM
        assert "static maximum" in htlr.htlr_last_error()
        assert lib.htlr_matvec_noalloc(None, u.data_ptr(), f.data_ptr(), 1) == htlr.HTLR_EINVAL
    finally:
        htlr.htlr_free(H)
