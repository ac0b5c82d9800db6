"""GMRES on the second-kind equation a(x) u + K u = f with HMultVec as the operator.

The solution is checked independently: the CPU oracle applies its own HTLR operator
(Algorithms 1-2, equal to the GPU operator to ~1e-14) to the GPU solution, and the
residual against f must reach the solver's tolerance."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _solve(w, f, far=0, near=0, inner=None, tol=1e-10, restart=30):
    import torch
    from paper_2508_05958_gb300 import htlr
    H = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, a=w.a(), far_precision=far,
                            near_precision=near)
    Hi = None
    if inner is not None:
        Hi = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, a=w.a(),
                                 far_precision=inner[0], near_precision=inner[1])
    try:
        fd = torch.from_numpy(np.ascontiguousarray(f.T)).cuda()
        ud = torch.zeros_like(fd)
        res = htlr.htlr_gmres(H, fd, ud, f.shape[1], H_inner=Hi, tol=tol, restart=restart)
        return ud.cpu().numpy().T.copy(), res
    finally:
        htlr.htlr_free(H)
        if Hi:
            htlr.htlr_free(Hi)


def _oracle_residual(oracle, w, u, f):
    Ho = oracle.HTLR(w.d, w.n, w.ktype, w.leaf, w.p, w.eta, a=w.a())
    r = f - Ho.matvec(u)
    return max(np.linalg.norm(r[:, c]) / np.linalg.norm(f[:, c]) for c in range(f.shape[1]))


def test_gmres_fp64_c1(oracle):
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c1")
    f = w.u(nrhs=3, seed=41)
    u, res = _solve(w, f)
    assert res["converged"] == 1 and res["rel_residual"] <= 1e-10
    assert res["refinements"] == 0 and res["iterations"] > 1
    assert _oracle_residual(oracle, w, u, f) < 2e-10


def test_gmres_small_restart_c2(oracle):
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2")
    f = w.u(nrhs=1, seed=42)
    u, res = _solve(w, f, far=1, near=1, restart=5)
    assert res["converged"] == 1
    assert _oracle_residual(oracle, w, u, f) < 2e-10


def test_gmres_mixed_precision_refinement_recovers_1e10(oracle):
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2")
    f = w.u(nrhs=2, seed=43)
    u, res = _solve(w, f, far=1, near=1, inner=(2, 1))
    assert res["converged"] == 1 and res["refinements"] >= 1
    assert _oracle_residual(oracle, w, u, f) < 2e-10


def test_gmres_rejects_bad_options():
    import torch
    from paper_2508_05958_gb300 import htlr
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c1", n=32)
    H = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, a=w.a())
    try:
        f = torch.zeros((1, w.N), dtype=torch.float64, device="cuda")
        u = torch.zeros_like(f)
        with pytest.raises(htlr.HTLRError):
            htlr.htlr_gmres(H, f, u, 1, restart=0)
        res = htlr.htlr_gmres(H, f, u, 1)            # f = 0: u = 0 is exact
        assert res["converged"] == 1 and float(u.abs().max()) == 0.0
    finally:
        htlr.htlr_free(H)
