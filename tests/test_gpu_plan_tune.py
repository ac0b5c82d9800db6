"""Matvec plans (CUDA graphs) and the launch-shape autotuner, through the C ABI.

A plan replays the exact launch sequence of htlr_matvec, so its result is bitwise equal.
The autotuner changes only launch shapes (task size, grid, ring depth), so results stay
within rounding of the untuned operator and within the FP64 bar (1e-12) of the CPU HTLR.
"""
import numpy as np
import pytest

from _helpers import rel

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_05958_gb300 import htlr
    htlr.load()


def _construct(w, **kw):
    from paper_2508_05958_gb300 import htlr
    return htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, kscale=w.kscale,
                               kparam=w.kparam, a=w.a(), **kw)


def _dev(u):
    import torch
    return torch.from_numpy(np.ascontiguousarray(u.T)).cuda()


def test_plan_replays_matvec_bitwise_and_follows_buffer_contents():
    import torch
    from paper_2508_05958_gb300 import htlr
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2")
    H = _construct(w, storage=1, far_precision=1, near_precision=1)
    try:
        u1, u2 = w.u(nrhs=3), w.u(nrhs=3, seed=77)
        ud = _dev(u1)
        f_ref = torch.empty_like(ud)
        htlr.htlr_matvec(H, ud, f_ref)
        fp = torch.full_like(ud, float("nan"))
        P = htlr.htlr_plan_create(H, ud, fp)
        try:
            assert htlr.htlr_plan_launches(P) >= 4
            htlr.htlr_plan_launch(P)
            htlr.htlr_sync(H)
            assert torch.equal(fp, f_ref)
            # new contents in the same buffer, replayed twice
            ud.copy_(_dev(u2))
            htlr.htlr_matvec(H, ud, f_ref)
            for _ in range(2):
                fp.fill_(float("nan"))
                htlr.htlr_plan_launch(P)
            htlr.htlr_sync(H)
            assert torch.equal(fp, f_ref)
        finally:
            htlr.htlr_plan_free(P)
    finally:
        htlr.htlr_free(H)


def test_plan_on_c1_against_oracle(oracle):
    import torch
    from paper_2508_05958_gb300 import htlr
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c1")
    u = w.u()
    H = _construct(w)
    try:
        ud = _dev(u)
        fd = torch.empty_like(ud)
        P = htlr.htlr_plan_create(H, ud, fd)
        htlr.htlr_plan_launch(P)
        htlr.htlr_sync(H)
        htlr.htlr_plan_free(P)
        f = fd.cpu().numpy().T
    finally:
        htlr.htlr_free(H)
    Ho = oracle.HTLR(w.d, w.n, w.ktype, w.leaf, w.p, w.eta, a=w.a())
    assert rel(f, Ho.matvec(u)) < TOL


def test_plan_rejects_bad_arguments():
    import torch
    from paper_2508_05958_gb300 import htlr
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c1")
    H = _construct(w)
    try:
        ud = _dev(w.u())
        with pytest.raises(htlr.HTLRError) as e:
            htlr.htlr_plan_create(H, ud, ud)      # u and f overlap
        assert e.value.code == htlr.HTLR_EINVAL
        with pytest.raises(htlr.HTLRError):
            htlr.htlr_plan_create(H, ud, torch.empty_like(ud), 0)
    finally:
        htlr.htlr_free(H)


@pytest.mark.parametrize("far,near,storage", [(1, 1, 1), (0, 0, 2), (2, 1, 1)])
def test_autotune_keeps_results_and_caches(oracle, far, near, storage):
    import torch
    from paper_2508_05958_gb300 import htlr
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2")
    htlr.htlr_autotune_clear_cache()
    u = w.u(nrhs=2)
    H = _construct(w, storage=storage, far_precision=far, near_precision=near)
    try:
        ud = _dev(u)
        f0 = torch.empty_like(ud)
        htlr.htlr_matvec(H, ud, f0)
        P = htlr.htlr_plan_create(H, ud, torch.empty_like(ud))
        r = htlr.htlr_autotune(H, nrhs=2, budget_ms=400.0)
        assert r["candidates"] >= 2 and r["from_cache"] == 0
        assert r["ms"] <= r["default_ms"] * 1.02
        assert r["task_bytes"] in (64 << 10, 128 << 10, 256 << 10, 512 << 10, 1024 << 10)
        assert r["stream_threads"] in (128, 256) and 2 <= r["stream_ctas_per_sm"] <= 16
        f1 = torch.empty_like(ud)
        htlr.htlr_matvec(H, ud, f1)
        htlr.htlr_plan_launch(P)          # re-captures if the task tables changed
        htlr.htlr_sync(H)
        htlr.htlr_plan_free(P)
        a, b = f0.cpu().numpy().T, f1.cpu().numpy().T
        # re-tasking changes only the order in which a row's partial sums are formed:
        # rounding of the stream's own precision (FP64, df64 ~1e-15, FP32 ~1e-7)
        assert rel(b, a) < {0: 1e-14, 1: 1e-13, 2: 1e-6}[far]
        H2 = _construct(w, storage=storage, far_precision=far, near_precision=near)
        try:
            r2 = htlr.htlr_autotune(H2, nrhs=2, budget_ms=400.0)
            assert r2["from_cache"] == 1 and r2["candidates"] == 0
            assert (r2["task_bytes"], r2["stream_ctas_per_sm"], r2["stream_threads"]) == (
                r["task_bytes"], r["stream_ctas_per_sm"], r["stream_threads"])
        finally:
            htlr.htlr_free(H2)
    finally:
        htlr.htlr_free(H)
    if far in (0, 1) and near in (0, 1):
        Ho = oracle.HTLR(w.d, w.n, w.ktype, w.leaf, w.p, w.eta, a=w.a())
        assert rel(b, Ho.matvec(u)) < TOL


def test_autotune_zero_budget_times_current_shapes_only():
    from paper_2508_05958_gb300 import htlr
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c1")
    htlr.htlr_autotune_clear_cache()
    H = _construct(w)
    try:
        r = htlr.htlr_autotune(H, nrhs=1, budget_ms=0.0)
        assert r["candidates"] == 1 and r["task_bytes"] == 256 << 10
    finally:
        htlr.htlr_free(H)


def test_autotune_tensor_core_ring_depth(oracle):
    import torch
    from paper_2508_05958_gb300 import htlr
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c1")
    htlr.htlr_autotune_clear_cache()
    u = w.u(nrhs=8)
    H = _construct(w, storage=2, far_precision=3, near_precision=3)
    try:
        ud = _dev(u)
        f0 = torch.empty_like(ud)
        htlr.htlr_matvec(H, ud, f0)
        r = htlr.htlr_autotune(H, nrhs=8, budget_ms=200.0)
        assert r["tc_stages"] in (0, 2, 3, 4)
        f1 = torch.empty_like(ud)
        htlr.htlr_matvec(H, ud, f1)
        htlr.htlr_sync(H)
        # the ring depth does not change the MMA order: identical results
        assert torch.equal(f0, f1)
    finally:
        htlr.htlr_free(H)
