"""Continuous-batching solve server on the GPU (htlr_server_*).

Bar: every request converges to the stated relative residual (1e-10, against the FP64
or df64 operator), a request's solution is the same alone and in a mix of concurrent
requests of several operators (stated tolerance 1e-12 relative; the batched matvec
computes each column as it would alone, so it is in fact expected bitwise), the server's
solution agrees with htlr_gmres on the same operator, and the residual re-checked with
the CPU oracle's HTLR operator meets the bar as well.
"""
import math

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SAME_TOL = 1e-12
WAIT_S = 300.0


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_05958_gb300 import htlr
    htlr.load()


def _ops():
    from paper_2508_05958_gb300.serving import OpSpec
    from paper_2508_05958_gb300.workloads import K_EXP_R, K_INV_R, K_LOG
    return [OpSpec(2, 64, K_LOG, 6, 8, math.sqrt(2.0), "one"),
            OpSpec(3, 16, K_INV_R, 5, 4, 1.0, "sin"),
            OpSpec(3, 32, K_EXP_R, 5, 4, 1.0, "sin")]


def _rhs(spec, seed):
    return np.random.default_rng(seed).standard_normal(spec.N)


def _solve(server, ops, jobs, op_ids=None):
    """Submit all jobs [(op, seed)] at once; return solutions and infos in job order."""
    if op_ids is None:
        op_ids = [server.add_operator(s.ktype, s.d, s.n, s.leaf, s.r, s.eta, a=s.a(), storage=2)
                  for s in ops]
    ids = [server.submit(op_ids[i], _rhs(ops[i], seed)) for i, seed in jobs]
    out = [server.wait(r, WAIT_S) for r in ids]
    return [u for u, _ in out], [inf for _, inf in out]


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("mixed,inner", [(0, 0), (1, 2)])
def test_mix_equals_alone_and_converges(mixed, inner):
    from paper_2508_05958_gb300 import htlr
    ops = _ops()
    jobs = [(i, 1000 + 10 * i + j) for j in range(3) for i in range(3)]
    with htlr.Server(mixed=mixed, inner_precision=inner, max_batch=8) as S:
        us, infos = _solve(S, ops, jobs)
        st = S.stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["max_batch_seen"] >= 2          # requests of one operator shared launches
    for inf in infos:
        assert inf["status"] == htlr.REQ_DONE and inf["converged"] == 1
        assert inf["rel_residual"] <= 1e-10
        if mixed:
            assert inf["refinements"] >= 1
    # each job alone: one request at a time on a fresh server
    with htlr.Server(mixed=mixed, inner_precision=inner, max_batch=8, max_active=1) as S1:
        ids = [S1.add_operator(s.ktype, s.d, s.n, s.leaf, s.r, s.eta, a=s.a(), storage=2)
               for s in ops]
        for k, (i, seed) in enumerate(jobs):
            u1, inf1 = _solve(S1, ops, [(i, seed)], op_ids=ids)
            assert inf1[0]["iterations"] == infos[k]["iterations"]
            assert _rel(us[k], u1[0]) <= SAME_TOL


def test_server_matches_htlr_gmres_and_oracle_residual(oracle):
    import torch
    from paper_2508_05958_gb300 import htlr
    ops = _ops()
    s = ops[0]
    f = _rhs(s, 7)
    with htlr.Server(mixed=0) as S:
        (u,), (inf,) = _solve(S, ops[:1], [(0, 7)])
    assert inf["converged"] == 1
    H = htlr.htlr_construct(s.ktype, s.d, s.n, s.leaf, s.r, s.eta, a=s.a(), storage=2)
    try:
        fd = torch.from_numpy(f).cuda()
        ud = torch.zeros_like(fd)
        res = htlr.htlr_gmres(H, fd, ud, 1)
        assert res["converged"]
        ug = ud.cpu().numpy()
    finally:
        htlr.htlr_free(H)
    assert _rel(u, ug) < 1e-8
    # the residual of the served solution under the CPU oracle's HTLR operator
    Ho = oracle.HTLR(s.d, s.n, s.ktype, s.leaf, s.r, s.eta, a=s.a())
    r = f - Ho.matvec(u.reshape(-1, 1))[:, 0]
    assert np.linalg.norm(r) / np.linalg.norm(f) < 2e-10


def test_tensor_core_inner_operator_converges():
    from paper_2508_05958_gb300 import htlr
    ops = _ops()[1:]
    jobs = [(i, 50 + 7 * i + j) for j in range(2) for i in range(2)]
    with htlr.Server(mixed=1, inner_precision=htlr.PREC_BF16X6, inner_tol=1e-3) as S:
        _, infos = _solve(S, ops, jobs)
    for inf in infos:
        assert inf["converged"] == 1 and inf["rel_residual"] <= 1e-10
        assert inf["refinements"] >= 1


def test_admission_by_footprint_evicts_idle_operators():
    from paper_2508_05958_gb300 import htlr
    ops = _ops()[1:]           # two d=3 operators
    m, batch = 30, 4
    foot = []
    for s in ops:
        H = htlr.htlr_construct(s.ktype, s.d, s.n, s.leaf, s.r, s.eta, a=s.a(), storage=2)
        foot.append(htlr.htlr_info(H)["bytes_total"] + 2 * 8 * s.N * batch)
        htlr.htlr_free(H)
    ws = max((m + 4) * 8 * s.N for s in ops)
    budget = max(foot) + 2 * ws + (1 << 20)
    assert budget < sum(foot) + 2 * ws          # both operators never fit together
    jobs = [(j % 2, 300 + j) for j in range(6)]
    with htlr.Server(mixed=0, max_batch=batch, hbm_budget=budget) as S:
        _, infos = _solve(S, ops, jobs)
        st = S.stats()
    assert all(inf["converged"] == 1 for inf in infos)
    # the second operator waits until the first one's requests are done, then replaces it
    assert st["evictions"] >= 1 and st["constructions"] >= 2
    assert st["resident_operators"] == 1
    assert st["bytes_peak"] <= budget


def test_request_that_cannot_fit_fails_without_blocking_others():
    from paper_2508_05958_gb300 import htlr
    ops = _ops()
    with htlr.Server(mixed=0, hbm_budget=1 << 20) as S:
        op = S.add_operator(ops[2].ktype, 3, 32, 4, 5, 1.0, a=ops[2].a(), storage=2)
        rid = S.submit(op, _rhs(ops[2], 1))
        _, inf = S.wait(rid, WAIT_S)
        assert inf["status"] == htlr.REQ_FAILED and inf["error"] == htlr.HTLR_ENOMEM
        with pytest.raises(htlr.HTLRError) as e:
            S.submit(17, _rhs(ops[2], 1))
        assert e.value.code == htlr.HTLR_EINVAL
        assert S.stats()["failed"] == 1


def test_batches_that_grow_and_shrink_between_steps():
    """Requests of one operator arriving in waves, so consecutive steps of the operator
    have batches of different sizes (the descriptors of one step must not disturb the
    copies of the previous one).  Every result equals its solo solve."""
    import time
    from paper_2508_05958_gb300 import htlr
    ops = _ops()[1:2]
    seeds = list(range(900, 924))
    with htlr.Server(mixed=1, inner_precision=htlr.PREC_FP32, max_batch=8) as S:
        op = S.add_operator(ops[0].ktype, ops[0].d, ops[0].n, ops[0].leaf, ops[0].r,
                            ops[0].eta, a=ops[0].a(), storage=2)
        ids = []
        for wave in range(6):
            for sd in seeds[4 * wave:4 * wave + 4]:
                ids.append(S.submit(op, _rhs(ops[0], sd)))
            time.sleep(0.002 * (wave % 3))
        out = [S.wait(r, WAIT_S) for r in ids]
        st = S.stats()
    assert st["completed"] == len(seeds) and st["failed"] == 0
    with htlr.Server(mixed=1, inner_precision=htlr.PREC_FP32, max_batch=8, max_active=1) as S1:
        op1 = S1.add_operator(ops[0].ktype, ops[0].d, ops[0].n, ops[0].leaf, ops[0].r,
                              ops[0].eta, a=ops[0].a(), storage=2)
        for (u, inf), sd in zip(out, seeds):
            assert inf["converged"] == 1
            u1, _ = S1.wait(S1.submit(op1, _rhs(ops[0], sd)), WAIT_S)
            assert _rel(u, u1) <= SAME_TOL
