"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bar: FP64 mode matches the oracle's HTLR (Algorithms 1-2) to a per-RHS relative 2-norm
of 1e-12 (the tolerance stated for FP64 mode), and the dense Nystrom product to the
interpolation accuracy; integer structure (block counts) is compared exactly.
"""
import math

import numpy as np
import pytest

from _helpers import gpu_matvec, rel

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2508_05958_gb300 import htlr
    htlr.load()


def _oracle_htlr(oracle, w, u, **kw):
    args = dict(a=w.a(), scale=w.kscale, param=w.kparam)
    args.update(kw)
    H = oracle.HTLR(w.d, w.n, args.pop("ktype", w.ktype), args.pop("leaf", w.leaf),
                    args.pop("p", w.p), args.pop("eta", w.eta), **args)
    return H.matvec(u), H.stats()


def test_c1_full_against_oracle_and_dense(oracle):
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c1")
    u = w.u()
    f, info = gpu_matvec(w, u)
    ref, st = _oracle_htlr(oracle, w, u)
    assert info["far_per_level"] == st[0] and info["near_blocks"] == st[1]
    assert rel(f, ref) < TOL
    fd = oracle.dense_rows(w.d, w.n, w.ktype, u, a=w.a())
    assert rel(f, fd) < 1e-6


def test_c2_full_against_oracle_and_dense(oracle):
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2")
    u = w.u()
    f, info = gpu_matvec(w, u, storage=1)
    assert info["storage"] == 1 and info["p_eff_leaf"] == 4
    ref, st = _oracle_htlr(oracle, w, u)
    assert info["far_per_level"] == st[0] == [0, 0, 1416, 133944]
    assert info["near_blocks"] == st[1] == 37576
    assert abs(info["paper_storage_doubles"] - st[2]) < 0.5
    assert rel(f, ref) < TOL
    rows = w.sample_rows(512)
    fd = oracle.dense_rows(w.d, w.n, w.ktype, u, rows=rows, a=w.a())
    assert rel(f[rows], fd) < 1e-6


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("case", [
    dict(d=2, n=32, leaf=4, p=4, eta=math.sqrt(2)),
    dict(d=2, n=64, leaf=8, p=3, eta=0.0),
    dict(d=3, n=16, leaf=4, p=3, eta=1.0),
    dict(d=3, n=16, leaf=2, p=3, eta=0.0),      # wide leaf factors: p_eff = 2 < p
    dict(d=3, n=8, leaf=4, p=2, eta=1.0),       # one level below the root
])
def test_polynomial_kernel_exact(oracle, case, storage):
    """Per-dimension degree p-1 is reproduced exactly: GPU == dense product."""
    from paper_2508_05958_gb300.workloads import Workload
    w = Workload("poly", d=case["d"], n=case["n"], ktype=4, leaf=case["leaf"], p=case["p"],
                 eta=case["eta"], kparam=case["p"] - 1, a_kind="one", seed=21)
    u = w.u(nrhs=3)
    f, info = gpu_matvec(w, u, storage=storage)
    assert info["storage"] == storage
    fd = oracle.dense_rows(w.d, w.n, 4, u, param=w.kparam, a=w.a())
    assert rel(f, fd) < 1e-13
    ref, _ = _oracle_htlr(oracle, w, u)
    assert rel(f, ref) < TOL


@pytest.mark.parametrize("orth", [0, 1])
@pytest.mark.parametrize("storage", [1, 2])
def test_orth_and_storage_modes_match_oracle(oracle, orth, storage):
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2", n=16, leaf=2, p=4)
    u = w.u(nrhs=2)
    f, _ = gpu_matvec(w, u, storage=storage, orth=orth)
    ref, _ = _oracle_htlr(oracle, w, u, orth=bool(orth))
    assert rel(f, ref) < TOL


@pytest.mark.parametrize("nrhs", [1, 2, 4, 5, 9])
def test_multi_rhs_chunks_and_ragged_tail(oracle, nrhs):
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c1", n=32)
    u = w.u(nrhs=nrhs)
    f, _ = gpu_matvec(w, u)
    ref, _ = _oracle_htlr(oracle, w, u)
    assert f.shape == (w.N, nrhs)
    assert rel(f, ref) < TOL


@pytest.mark.parametrize("ktype,kscale,kparam", [(0, -1 / (2 * math.pi), 0.0), (2, 1.0, 0.0),
                                                 (3, 1.0, math.sqrt(2)), (5, 0.7, 0.0)])
def test_other_kernels_2d(oracle, ktype, kscale, kparam):
    from paper_2508_05958_gb300.workloads import Workload
    w = Workload("k", d=2, n=64, ktype=ktype, leaf=8, p=5, eta=math.sqrt(2), kscale=kscale,
                 kparam=kparam, a_kind="one", seed=5)
    u = w.u(nrhs=1)
    f, _ = gpu_matvec(w, u)
    ref, _ = _oracle_htlr(oracle, w, u)
    assert rel(f, ref) < TOL


def test_weak_admissibility_3d_gaussian(oracle):
    from paper_2508_05958_gb300.workloads import Workload
    w = Workload("g", d=3, n=32, ktype=3, leaf=4, p=4, eta=0.0, kparam=math.sqrt(3), seed=6)
    u = w.u(nrhs=1)
    f, info = gpu_matvec(w, u)
    ref, st = _oracle_htlr(oracle, w, u)
    assert info["far_per_level"] == st[0]
    assert rel(f, ref) < TOL


def test_host_entry_point_and_determinism(oracle):
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2", n=16, leaf=4)
    u = w.u(nrhs=3)
    outs, _ = gpu_matvec(w, u, repeat=3)
    assert all(np.array_equal(outs[0], o) for o in outs[1:])     # bitwise repeatable
    fh, _ = gpu_matvec(w, u, host=True)
    assert np.array_equal(fh, outs[0])


def test_diagonal_value_matches_closed_form():
    from paper_2508_05958_gb300 import htlr
    h = 1.0 / 32
    H = htlr.htlr_construct(1, 3, 32, 4, 5, 1.0)
    try:
        dv = htlr.htlr_info(H)["diag_value"]
    finally:
        htlr.htlr_free(H)
    exact = (3 * math.log(2 + math.sqrt(3)) - math.pi / 2) * h * h
    assert abs(dv - exact) < 2e-5 * exact


def test_memory_limit_refusal():
    from paper_2508_05958_gb300 import htlr
    with pytest.raises(htlr.HTLRError) as ei:
        htlr.htlr_construct(1, 3, 32, 4, 5, 1.0, storage=1, hbm_limit=1 << 20)
    assert ei.value.code == htlr.HTLR_ENOMEM


# ----------------------------------------------------------------------------------
# Precisions: df64 (FP64 accuracy through FP32 pairs) meets the FP64 tolerance; the FP32
# far field meets the mixed-precision tolerance (1e-6 relative, stated for that mode).
# ----------------------------------------------------------------------------------
MIXED_TOL = 1e-6
FP32_TOL = 1e-5     # far and near fields both in FP32
# tensor cores (three-way BF16 split, FP32 accumulation in tensor memory): the products
# are FP32-class, and the tensor cores truncate every addition to the accumulator.  The
# grouped kernel starts each segment of two K steps from a fresh accumulator with the
# small cross products first, and adds the segments in FP32 registers that are flushed to
# FP64 every 32 segments: a stated tolerance of 1e-6 relative.
TC_TOL = 1e-6


@pytest.mark.parametrize("storage", [1, 2])
@pytest.mark.parametrize("name", ["c1", "c2"])
def test_df64_meets_fp64_tolerance(oracle, name, storage):
    from paper_2508_05958_gb300.workloads import workload
    w = workload(name)
    u = w.u(nrhs=2)
    f, info = gpu_matvec(w, u, storage=storage, far_precision=1, near_precision=1)
    assert info["far_precision"] == 1 and info["near_precision"] == 1
    ref, _ = _oracle_htlr(oracle, w, u)
    assert rel(f, ref) < TOL


@pytest.mark.parametrize("near", [0, 1])
@pytest.mark.parametrize("storage", [1, 2])
def test_fp32_far_field_mixed_tolerance(oracle, near, storage):
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2")
    u = w.u(nrhs=1)
    f, info = gpu_matvec(w, u, storage=storage, far_precision=2, near_precision=near)
    ref, _ = _oracle_htlr(oracle, w, u)
    err = rel(f, ref)
    assert err < MIXED_TOL, err
    assert err > 1e-12                      # it is genuinely FP32 arithmetic


def test_df64_polynomial_exactness_and_determinism(oracle):
    from paper_2508_05958_gb300.workloads import Workload
    w = Workload("poly", d=3, n=16, ktype=4, leaf=2, p=3, eta=1.0, kparam=2, a_kind="one", seed=22)
    u = w.u(nrhs=3)
    outs, _ = gpu_matvec(w, u, far_precision=1, near_precision=1, repeat=2)
    assert np.array_equal(outs[0], outs[1])
    fd = oracle.dense_rows(w.d, w.n, 4, u, param=2, a=w.a())
    assert rel(outs[0], fd) < 1e-12


# ----------------------------------------------------------------------------------
# Tensor (quasi-uniform) grids and the generated near field
# ----------------------------------------------------------------------------------
def _qgrid(d, n, seed=5):
    from paper_2508_05958_gb300.workloads import quasi_uniform_tensor_grid
    return quasi_uniform_tensor_grid(d, n, seed)


def _gpu_tensor(w, grid, u, a=None, **kw):
    import torch
    from paper_2508_05958_gb300 import htlr
    H = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, kscale=w.kscale,
                            kparam=w.kparam, a=a, grid=grid, **kw)
    try:
        info = htlr.htlr_info(H)
        nr = u.shape[1]
        ud = torch.from_numpy(np.ascontiguousarray(u.T)).cuda()
        fd = torch.full_like(ud, float("nan"))
        htlr.htlr_matvec(H, ud, fd, nr)
        htlr.htlr_sync(H)
        return fd.cpu().numpy().T.copy(), info
    finally:
        htlr.htlr_free(H)


@pytest.mark.parametrize("d,n,leaf,p,eta", [(2, 32, 4, 4, 1.0), (3, 16, 4, 3, 1.0),
                                            (3, 16, 2, 3, 0.0)])
def test_tensor_grid_polynomial_exact(oracle, d, n, leaf, p, eta):
    from paper_2508_05958_gb300.workloads import Workload
    w = Workload("tp", d=d, n=n, ktype=4, leaf=leaf, p=p, eta=eta, kparam=p - 1, seed=31)
    grid = _qgrid(d, n)
    u = w.u(nrhs=2)
    a = np.random.default_rng(3).uniform(0.5, 1.5, w.N)
    f, info = _gpu_tensor(w, grid, u, a=a)
    assert info["storage"] == 3
    fd = oracle.dense_rows(d, n, 4, u, param=p - 1, a=a, grid=grid)
    assert rel(f, fd) < 1e-12


@pytest.mark.parametrize("ktype", [2, 1])
def test_tensor_grid_matches_oracle_htlr(oracle, ktype):
    from paper_2508_05958_gb300.workloads import Workload
    w = Workload("tq", d=3, n=32, ktype=ktype, leaf=4, p=4, eta=1.0, seed=32)
    grid = _qgrid(3, 32, seed=7)
    u = w.u(nrhs=3)
    f, info = _gpu_tensor(w, grid, u)
    H = oracle.HTLR(3, 32, ktype, 4, 4, 1.0, grid=grid, orth=False)
    ref = H.matvec(u)
    assert info["far_per_level"] == H.stats()[0]
    assert rel(f, ref) < TOL
    # mixed precision (FP32 far field, FP64 near field) stays within the mixed tolerance;
    # with the generated near field in FP32 too, within the looser FP32 bound
    fmix, _ = _gpu_tensor(w, grid, u, far_precision=2, near_precision=0)
    assert rel(fmix, ref) < MIXED_TOL
    f32, _ = _gpu_tensor(w, grid, u, far_precision=2, near_precision=2)
    assert rel(f32, ref) < FP32_TOL


@pytest.mark.parametrize("nrhs", [1, 3, 9])
def test_tensor_grid_large_leaves_generated_near(oracle, nrhs):
    """Leaves of 7-9 points per dimension (up to 729 rows: three target rows per thread
    in the generated near field) at every RHS count class of that kernel."""
    from paper_2508_05958_gb300.workloads import Workload
    w = Workload("tl", d=3, n=32, ktype=2, leaf=8, p=5, eta=1.0, seed=34)
    grid = _qgrid(3, 32, seed=9)
    u = w.u(nrhs=nrhs)
    f, info = _gpu_tensor(w, grid, u)
    assert info["storage"] == 3
    H = oracle.HTLR(3, 32, 2, 8, 5, 1.0, grid=grid, orth=False)
    ref = H.matvec(u)
    assert rel(f, ref) < TOL
    f32, _ = _gpu_tensor(w, grid, u, far_precision=2, near_precision=2)
    assert rel(f32, ref) < FP32_TOL


@pytest.mark.parametrize("near", [0, 2])
def test_uniform_generated_near_field(oracle, near):
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2", n=16)
    u = w.u(nrhs=5)
    f, info = gpu_matvec(w, u, storage=3, near_precision=near)
    assert info["storage"] == 3 and info["unique_near"] == 0
    ref, _ = _oracle_htlr(oracle, w, u)
    assert rel(f, ref) < (TOL if near == 0 else FP32_TOL)


def test_tensor_grid_rejects_empty_boxes_and_orth():
    from paper_2508_05958_gb300 import htlr
    x = np.tile((np.arange(8) + 0.5) / 8, (2, 1))
    x[0] = np.linspace(0.01, 0.3, 8)              # nothing in the upper half of dim 1
    e = np.zeros((2, 9))
    for l in range(2):
        e[l, 1:8] = 0.5 * (x[l, :-1] + x[l, 1:])
        e[l, 8] = 1.0
    with pytest.raises(htlr.HTLRError) as ei:
        htlr.htlr_construct(2, 2, 8, 2, 3, 1.0, grid=(x, e))
    assert ei.value.code == htlr.HTLR_EINVAL
    g = _qgrid(2, 16)
    with pytest.raises(htlr.HTLRError) as ei:
        htlr.htlr_construct(2, 2, 16, 4, 3, 1.0, grid=g, orth=1)
    assert ei.value.code == htlr.HTLR_EUNSUPPORTED


# ----------------------------------------------------------------------------------
# Tensor cores (tcgen05, three-way BF16 split, FP32 accumulation) for many right-hand sides
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("nrhs", [1, 16, 20, 64, 70])
def test_tensor_core_stream_matches_oracle(oracle, nrhs):
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2", n=16)                      # 125-row cores (pe = 5) and 64-row leaves
    u = w.u(nrhs=nrhs)
    f, info = gpu_matvec(w, u, storage=2, far_precision=3, near_precision=3)
    assert info["far_precision"] == 3
    # SHARED: every far level and the leaves on the target-grouped kernel
    want = sum(1 << lv for lv, c in enumerate(info["far_per_level"]) if c) - (1 << 31)
    assert info["tc_grouped"] == want
    ref, _ = _oracle_htlr(oracle, w, u)
    err = rel(f, ref)
    assert err < TC_TOL, err


def test_tensor_core_refuses_stored_blocks():
    """BF16X6 block lists are held one block per (level, offset), where the grouped kernel
    reads each block once per group of targets; STORED blocks are refused explicitly and
    AUTO resolves to SHARED."""
    from paper_2508_05958_gb300 import htlr
    with pytest.raises(htlr.HTLRError) as ei:
        htlr.htlr_construct(1, 3, 16, 4, 5, 1.0, storage=1, far_precision=3, near_precision=3)
    assert ei.value.code == htlr.HTLR_EUNSUPPORTED
    H = htlr.htlr_construct(1, 3, 16, 4, 5, 1.0, storage=0, far_precision=3, near_precision=3)
    try:
        assert htlr.htlr_info(H)["storage"] == 2
    finally:
        htlr.htlr_free(H)


@pytest.mark.parametrize("seg,flush", [(1, 1), (1, 32), (4, 8), (2, 1000)])
def test_tensor_core_segments_change_only_rounding(oracle, seg, flush):
    """Segment length and flush interval change the order of the FP32 additions only:
    every setting stays within the tolerance, and repeated matvecs are bitwise equal."""
    import torch
    from paper_2508_05958_gb300 import htlr
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2", n=32, leaf=8, p=6, a_kind="zero")   # 216-row cores, 512-row leaves
    u = w.u(nrhs=16)
    ref, _ = _oracle_htlr(oracle, w, u)
    H = htlr.htlr_construct(w.ktype, w.d, w.n, w.leaf, w.p, w.eta, storage=2, far_precision=3,
                            near_precision=3, tc_segment=seg, tc_flush=flush)
    try:
        ud = torch.from_numpy(np.ascontiguousarray(u.T)).cuda()
        f1, f2 = torch.empty_like(ud), torch.empty_like(ud)
        htlr.htlr_matvec(H, ud, f1, 16)
        htlr.htlr_matvec(H, ud, f2, 16)
        htlr.htlr_sync(H)
        assert torch.equal(f1, f2)
        assert rel(f1.cpu().numpy().T, ref) < TC_TOL
    finally:
        htlr.htlr_free(H)


@pytest.mark.parametrize("case", [dict(name="c1", over={}), dict(name="c3", over=dict(n=32)),
                                  dict(name="c2", over=dict(n=32, leaf=8, p=6))])
def test_tensor_core_stream_shapes(oracle, case):
    """d = 2 (36-row cores), 216-row cores over two M-tiles, 512-row leaf blocks over four."""
    from paper_2508_05958_gb300.workloads import workload
    w = workload(case["name"], **case["over"])
    u = w.u(nrhs=8)
    f, _ = gpu_matvec(w, u, storage=2, far_precision=3, near_precision=3)
    ref, _ = _oracle_htlr(oracle, w, u)
    assert rel(f, ref) < TC_TOL


def test_tensor_core_far_with_generated_near(oracle):
    from paper_2508_05958_gb300.workloads import Workload
    w = Workload("tq", d=3, n=32, ktype=2, leaf=4, p=4, eta=1.0, seed=33)
    grid = _qgrid(3, 32, seed=9)
    u = w.u(nrhs=16)
    f, info = _gpu_tensor(w, grid, u, far_precision=3, near_precision=0)
    ref = oracle.HTLR(3, 32, 2, 4, 4, 1.0, grid=grid, orth=False).matvec(u)
    assert rel(f, ref) < TC_TOL


@pytest.mark.parametrize("storage,near,nrhs", [(2, 0, 16), (2, 1, 37), (0, 1, 8), (2, 2, 64)])
def test_tensor_core_far_with_held_cuda_core_near(oracle, storage, near, nrhs):
    """BF16-split far field on the tensor cores, held near field (FP64, df64 or FP32) on
    the CUDA cores in passes of four right-hand sides."""
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2", n=16)
    u = w.u(nrhs=nrhs)
    f, info = gpu_matvec(w, u, storage=storage, far_precision=3, near_precision=near)
    assert info["far_precision"] == 3 and info["near_precision"] == near
    ref, _ = _oracle_htlr(oracle, w, u)
    assert rel(f, ref) < TC_TOL


def test_tensor_core_rejects_unsupported_mixes():
    from paper_2508_05958_gb300 import htlr
    with pytest.raises(htlr.HTLRError) as ei:
        htlr.htlr_construct(1, 3, 16, 4, 4, 1.0, storage=2, far_precision=0, near_precision=3)
    assert ei.value.code == htlr.HTLR_EUNSUPPORTED
    # the TF32X3 near field is generated: refused with held dense blocks, and not a far field
    for storage in (1, 2):
        with pytest.raises(htlr.HTLRError) as ei:
            htlr.htlr_construct(1, 3, 16, 4, 4, 1.0, storage=storage, near_precision=4)
        assert ei.value.code == htlr.HTLR_EUNSUPPORTED
    for far, near in ((4, 0), (0, 5)):
        with pytest.raises(htlr.HTLRError) as ei:
            htlr.htlr_construct(1, 3, 16, 4, 4, 1.0, far_precision=far, near_precision=near)
        assert ei.value.code == htlr.HTLR_EINVAL


# ----------------------------------------------------------------------------------
# Generated near field on the tensor cores (TF32X3): kernel values generated per pair
# into tensor memory as two TF32 terms, times w u packed as two TF32 terms, 16 RHS a pass
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("ktype,kparam,nrhs", [(2, 0.0, 16), (1, 0.0, 5), (3, 0.3, 21),
                                               (0, 0.0, 16), (4, 2.0, 3)])
def test_tf32x3_generated_near_tensor_grid(oracle, ktype, kparam, nrhs):
    """Leaves of 7-9 points per dimension (343-729 rows: three to six 128-row tiles, the
    last one ragged), 16-source stages with a padded tail per source leaf, RHS counts of
    one full pass, one padded pass and two passes, and every branch of the generator
    (exp(-r) packed; 1/r; Gaussian; log; the polynomial test kernel)."""
    from paper_2508_05958_gb300.workloads import Workload
    w = Workload("tl", d=3, n=32, ktype=ktype, leaf=8, p=5, eta=1.0, kparam=kparam, seed=34)
    grid = _qgrid(3, 32, seed=9)
    u = w.u(nrhs=nrhs)
    f, info = _gpu_tensor(w, grid, u, far_precision=0, near_precision=4)
    assert info["storage"] == 3 and info["near_precision"] == 4
    ref = oracle.HTLR(3, 32, ktype, 8, 5, 1.0, grid=grid, orth=False, param=kparam).matvec(u)
    assert rel(f, ref) < TC_TOL


@pytest.mark.parametrize("storage", [0, 3])
def test_tf32x3_uniform_grid_generated(oracle, storage):
    """Uniform grid, 1/r with a(x) = 1 + sin (64-point leaves: one ragged tile); AUTO
    storage generates the near field when its precision is TF32X3."""
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2", n=16)
    u = w.u(nrhs=16)
    f, info = gpu_matvec(w, u, storage=storage, near_precision=4)
    assert info["storage"] == 3 and info["unique_near"] == 0
    ref, _ = _oracle_htlr(oracle, w, u)
    assert rel(f, ref) < TC_TOL


def test_tf32x3_2d_log_kernel(oracle):
    """2D single-layer potential, leaves of 16^2 = 256 points (two full tiles)."""
    from paper_2508_05958_gb300.workloads import Workload
    w = Workload("k", d=2, n=128, ktype=0, leaf=16, p=6, eta=math.sqrt(2),
                 kscale=-1 / (2 * math.pi), a_kind="one", seed=6)
    u = w.u(nrhs=16)
    f, info = gpu_matvec(w, u, storage=3, near_precision=4)
    ref, _ = _oracle_htlr(oracle, w, u)
    assert rel(f, ref) < TC_TOL


def test_tf32x3_near_with_tensor_core_far(oracle):
    """Both fields on the tensor cores: BF16X6 far (grouped kernel on the tensor grid's
    shared cores), TF32X3 generated near."""
    from paper_2508_05958_gb300.workloads import Workload
    w = Workload("tq", d=3, n=32, ktype=2, leaf=4, p=4, eta=1.0, seed=33)
    grid = _qgrid(3, 32, seed=9)
    u = w.u(nrhs=32)
    f, info = _gpu_tensor(w, grid, u, far_precision=3, near_precision=4)
    ref = oracle.HTLR(3, 32, 2, 4, 4, 1.0, grid=grid, orth=False).matvec(u)
    assert rel(f, ref) < TC_TOL


# ----------------------------------------------------------------------------------
# Degenerate settings of the method
# ----------------------------------------------------------------------------------
@pytest.mark.parametrize("storage,far,near", [(1, 0, 0), (2, 1, 1), (2, 3, 3)])
def test_nothing_admissible_is_the_dense_product(oracle, storage, far, near):
    """eta so small that no block is admissible (Def. 2.3: max diam <= eta dist never
    holds): the operator is its near field alone and equals the dense Nystrom product
    (same diagonal rule) on every row."""
    from paper_2508_05958_gb300.workloads import workload
    w = workload("c2", n=16)
    u = w.u(nrhs=3)
    f, info = gpu_matvec(w, u, eta=1e-9, storage=storage, far_precision=far, near_precision=near)
    assert sum(info["far_per_level"]) == 0
    assert info["near_blocks"] == (16 // 4) ** 6
    fd = oracle.dense_rows(w.d, w.n, w.ktype, u, a=w.a())
    assert rel(f, fd) < (TOL if near in (0, 1) else TC_TOL)


def test_single_level_tree_2d(oracle):
    """n = 2 leaf (one level below the root) with weak admissibility: four leaf boxes,
    every pair of distinct boxes admissible at level 1, only the diagonal blocks dense."""
    from paper_2508_05958_gb300.workloads import Workload
    w = Workload("t1", d=2, n=16, ktype=3, leaf=8, p=6, eta=0.0, kparam=0.7, seed=5)
    u = w.u(nrhs=2)
    f, info = gpu_matvec(w, u)
    assert info["far_per_level"] == [0, 12] and info["near_blocks"] == 4
    ref, _ = _oracle_htlr(oracle, w, u)
    assert rel(f, ref) < TOL


def test_zero_and_constant_inputs():
    """u = 0 gives f = 0 exactly; the constant kernel with a = 0 gives c h^d sum(u) in
    every row (all blocks rank one), to rounding."""
    import torch
    from paper_2508_05958_gb300 import htlr
    n, d = 16, 3
    N = n ** d
    H = htlr.htlr_construct(5, d, n, 4, 3, 1.0, kscale=2.5, storage=2)
    try:
        z = torch.zeros(2, N, dtype=torch.float64, device="cuda")
        fz = torch.full_like(z, float("nan"))
        htlr.htlr_matvec(H, z, fz)
        htlr.htlr_sync(H)
        assert torch.count_nonzero(fz).item() == 0
        u = torch.from_numpy(np.random.default_rng(1).standard_normal((1, N))).cuda()
        f = torch.empty_like(u)
        htlr.htlr_matvec(H, u, f)
        htlr.htlr_sync(H)
        expect = 2.5 * (1.0 / n) ** d * u.sum().item()
        # the diagonal entry of the constant kernel is its cell integral: c h^d as well
        assert torch.allclose(f, torch.full_like(f, expect), rtol=0, atol=1e-12 * abs(expect) + 1e-14)
    finally:
        htlr.htlr_free(H)


@pytest.mark.parametrize("case", [dict(n=512, leaf=8, p=6, eta=math.sqrt(2.0), k=0, sig=0.0),
                                  dict(n=1024, leaf=8, p=7, eta=math.sqrt(2.0), k=0, sig=0.0),
                                  dict(n=2048, leaf=16, p=8, eta=0.0, k=3, sig=math.sqrt(2.0))])
@pytest.mark.parametrize("prec", [0, 1])
def test_large_2d_boxes_match_oracle_rows(oracle, case, prec):
    """2D operators whose upper levels hold large boxes (128^2 to 1024^2 points): the
    upward and downward contractions stage their data in bounded pieces of shared
    memory.  FP64 and df64 against the oracle's row-sampled HTLR."""
    from paper_2508_05958_gb300.workloads import Workload
    w = Workload("big2d", d=2, n=case["n"], ktype=case["k"], leaf=case["leaf"], p=case["p"],
                 eta=case["eta"], kparam=case["sig"], a_kind="one", seed=51)
    u = w.u(nrhs=2)
    rows = w.sample_rows(12, seed=52)
    f, info = gpu_matvec(w, u, storage=2, far_precision=prec, near_precision=prec)
    ref = oracle.htlr_rows(w.d, w.n, w.ktype, w.leaf, w.p, w.eta, u, rows, param=w.kparam,
                           a=w.a())
    assert rel(f[rows], ref) < TOL


def test_tf32x3_largest_leaves_2d(oracle):
    """The largest leaves the library takes (32^2 = 1024 points: eight 128-row tiles, the
    largest coordinate buffer of the generating warpgroups), 2D Gaussian, with two passes
    of 16 RHS of which the second is padded."""
    from paper_2508_05958_gb300.workloads import Workload
    w = Workload("leaf32", d=2, n=256, ktype=3, leaf=32, p=6, eta=math.sqrt(2.0),
                 kparam=math.sqrt(2.0), a_kind="one", seed=53)
    u = w.u(nrhs=20)
    rows = w.sample_rows(24, seed=54)
    f, info = gpu_matvec(w, u, storage=3, near_precision=4)
    assert info["storage"] == 3 and info["near_precision"] == 4
    ref = oracle.htlr_rows(w.d, w.n, w.ktype, w.leaf, w.p, w.eta, u, rows, param=w.kparam,
                           a=w.a())
    assert rel(f[rows], ref) < TC_TOL
