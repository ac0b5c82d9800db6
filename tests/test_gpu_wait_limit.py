"""Failure detection of the tensor-core kernels without a GPU fault.

Every wait inside the tcgen05 kernels (for a copy, an MMA commit or a drained
accumulator) is bounded.  A handle built with a wait limit of a few SM cycles makes those
waits run out on purpose: a copy from HBM or a segment of MMAs takes thousands of cycles,
and limits that short poll without suspending.  The kernel must then stop, let what it
issued complete, free its tensor memory and return; the host must read HTLR_ETIMEOUT
from htlr_sync; and the same handle must work again, with a correct result, once the
default limit is restored.
"""
import numpy as np
import pytest

from _helpers import rel

pytestmark = pytest.mark.gpu

TC_TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_05958_gb300 import htlr
    htlr.load()


def test_short_wait_limit_times_out_and_the_handle_recovers(oracle):
    import torch
    from paper_2508_05958_gb300 import htlr
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2", n=16)                      # d=3, 1/r, leaf 4^3, p=5, eta=1
    nrhs = 16
    u = w.u(nrhs=nrhs)
    H = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, a=w.a(), storage=2,
                            far_precision=3, near_precision=3, tc_wait_cycles=8)
    try:
        info = htlr.htlr_info(H)
        # every block list on the grouped tensor-core kernel (the one under test)
        want = sum(1 << lv for lv, c in enumerate(info["far_per_level"]) if c) - (1 << 31)
        assert info["tc_grouped"] == want
        ud = torch.from_numpy(np.ascontiguousarray(u.T)).cuda()
        fd = torch.full_like(ud, float("nan"))
        htlr.htlr_matvec(H, ud, fd, nrhs)        # asynchronous: the error waits for sync
        with pytest.raises(htlr.HTLRError) as ei:
            htlr.htlr_sync(H)
        assert ei.value.code == htlr.HTLR_ETIMEOUT
        assert "ran out" in str(ei.value)
        # the report cleared the error word: the stream is idle and nothing new failed
        htlr.htlr_sync(H)
        # the same handle, default limit: a valid product again
        htlr.htlr_set_wait_limit(H, 0)
        fd.fill_(float("nan"))
        htlr.htlr_matvec(H, ud, fd, nrhs)
        htlr.htlr_sync(H)
        f = fd.cpu().numpy().T.copy()
    finally:
        htlr.htlr_free(H)
    ref = oracle.HTLR(w.d, w.n, w.ktype, w.leaf, w.p, w.eta, a=w.a()).matvec(u)
    assert rel(f, ref) < TC_TOL


def test_synchronous_entry_point_reports_the_timeout(oracle):
    """htlr_matvec_host waits for its copies, so it reads the error word itself."""
    from paper_2508_05958_gb300 import htlr
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2", n=16)
    u = np.asfortranarray(w.u(nrhs=16))
    f = np.zeros_like(u, order="F")
    H = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, a=w.a(), storage=2,
                            far_precision=3, near_precision=3, tc_wait_cycles=8)
    try:
        with pytest.raises(htlr.HTLRError) as ei:
            htlr.htlr_matvec_host(H, u, f, 16)
        assert ei.value.code == htlr.HTLR_ETIMEOUT
        htlr.htlr_set_wait_limit(H, 0)
        htlr.htlr_matvec_host(H, u, f, 16)
    finally:
        htlr.htlr_free(H)
    ref = oracle.HTLR(w.d, w.n, w.ktype, w.leaf, w.p, w.eta, a=w.a()).matvec(u)
    assert rel(f, ref) < TC_TOL


def test_wait_limit_rejects_negative():
    from paper_2508_05958_gb300 import htlr
    with pytest.raises(htlr.HTLRError) as ei:
        htlr.htlr_construct(1, 3, 16, 4, 4, 1.0, storage=2, far_precision=3, near_precision=3,
                            tc_wait_cycles=-1)
    assert ei.value.code == htlr.HTLR_EINVAL


def test_generated_near_field_on_tensor_cores_times_out_and_recovers(oracle):
    """The TF32X3 generated near field: its drains and its MMA thread wait with the same
    bounded limit."""
    import torch
    from paper_2508_05958_gb300 import htlr
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2", n=16)
    u = w.u(nrhs=16)
    H = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, a=w.a(), storage=3,
                            near_precision=4, tc_wait_cycles=8)
    try:
        ud = torch.from_numpy(np.ascontiguousarray(u.T)).cuda()
        fd = torch.full_like(ud, float("nan"))
        htlr.htlr_matvec(H, ud, fd, 16)
        with pytest.raises(htlr.HTLRError) as ei:
            htlr.htlr_sync(H)
        assert ei.value.code == htlr.HTLR_ETIMEOUT
        htlr.htlr_sync(H)
        htlr.htlr_set_wait_limit(H, 0)
        fd.fill_(float("nan"))
        htlr.htlr_matvec(H, ud, fd, 16)
        htlr.htlr_sync(H)
        f = fd.cpu().numpy().T.copy()
    finally:
        htlr.htlr_free(H)
    ref = oracle.HTLR(w.d, w.n, w.ktype, w.leaf, w.p, w.eta, a=w.a()).matvec(u)
    assert rel(f, ref) < TC_TOL
