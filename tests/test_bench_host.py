"""The benchmark's roofline arithmetic on the host: algorithmic bytes and multiply-adds
per launch follow from the block counts of the cluster tree (Def. 2.4, counted by the
oracle) and the element sizes of each precision; the bound and the fraction follow from
those and the launch time.  No device is used."""
import math

import numpy as np
import pytest

import bench
from paper_2508_05958_gb300.workloads import workload


def _info(w, storage, far, near, oracle):
    far_per_level, near_blocks, _ = oracle.htlr_count(w.d, w.n, w.leaf, w.p, w.eta)
    return {"far_per_level": far_per_level, "near_blocks": near_blocks, "storage": storage,
            "far_precision": far, "near_precision": near}


def test_c2_stored_elements_match_the_cluster_tree(oracle):
    w = workload("c2")
    info = _info(w, 1, 1, 1, oracle)
    assert info["far_per_level"] == [0, 0, 1416, 133944] and info["near_blocks"] == 37576
    far, near, far_u, near_u = bench.stream_elements(info, w)
    # level 2: boxes of 8 points per dimension, p_eff = 5; level 3: 4 points, p_eff = 4
    assert far == 1416 * 5 ** 6 + 133944 * 4 ** 6
    assert near == 37576 * 64 * 64
    assert (far_u, near_u) == (far, near)          # STORED holds every block


@pytest.mark.parametrize("far,near,bound", [(1, 1, "hbm"), (2, 1, "hbm"), (0, 0, "alu")])
def test_stream_roofline_bound_and_fraction(oracle, far, near, bound):
    w = workload("c2")
    info = _info(w, 1, far, near, oracle)
    ms, peak = 0.9, 6809.3
    roof = bench.stream_roofline(info, w, 1, ms, peak, "measured")
    fe, ne, _, _ = bench.stream_elements(info, w)
    nbytes = fe * bench.PREC_BYTES[far] + ne * bench.PREC_BYTES[near]
    assert roof["algorithmic_bytes_per_launch"] == nbytes
    assert roof["multiply_adds_per_launch"] == fe + ne
    assert roof["bound"] == bound
    if bound == "hbm":
        assert roof["achieved"] == pytest.approx(nbytes / (ms * 1e-3) / 1e9, rel=1e-12)
        assert roof["frac"] == pytest.approx(roof["achieved"] / peak, rel=1e-12)
    else:
        # FP64: 2 flops per multiply-add against 152 SMs x 2 FMA/clk x 2.07 GHz
        assert roof["peak"] == pytest.approx(2 * 152 * 2 * 2.07e9 / 1e12, rel=1e-12)
        assert roof["achieved"] == pytest.approx(2 * (fe + ne) / (ms * 1e-3) / 1e12, rel=1e-12)
    assert 0 < roof["frac"]


def test_df64_stored_c2_headline_bytes(oracle):
    """The default benchmark line: c2 STORED df64 streams 5,797,367,360 bytes per matvec
    (8 bytes per core or dense-block element)."""
    w = workload("c2")
    roof = bench.stream_roofline(_info(w, 1, 1, 1, oracle), w, 1, 1.0, 6809.3, "measured")
    assert roof["algorithmic_bytes_per_launch"] == 5797367360


def test_generated_near_roofline_counts_pairs_times_rhs():
    info = {"near_precision": 2, "storage": 3, "near_point_pairs": 10_000_000}
    roof = bench.near_cc_roofline(info, workload("c4"), 16, 2.0)
    assert roof["multiply_adds_per_launch"] == 16 * 10_000_000
    assert roof["achieved"] == pytest.approx(2 * 16e7 / 2e-3 / 1e12, rel=1e-12)
    assert roof["peak"] == pytest.approx(2 * 152 * 128 * 2.07e9 / 1e12, rel=1e-12)
    assert roof["kernel_evaluations_per_s"] == pytest.approx(1e7 / 2e-3, rel=1e-12)


@pytest.mark.parametrize("ktype,sfu", [(2, 2), (1, 1), (3, 1), (0, 1), (4, None)])
def test_tensor_core_near_roofline_is_the_sfu_rate(ktype, sfu):
    """The generated near field on the tensor cores: kernel values per second against
    152 SMs x 2.07 GHz x 16 SFU operations per clock, divided by the SFU operations one
    value costs (exp(-r): rsqrt and ex2; 1/r, the Gaussian, log: one); the polynomial
    test kernel uses none and has no SFU bound."""
    from paper_2508_05958_gb300.workloads import Workload
    w = Workload("k", d=3, n=16, ktype=ktype, leaf=4, p=3, eta=1.0)
    info = {"near_precision": 4, "storage": 3, "near_point_pairs": 2_000_000}
    roof = bench.near_tc_roofline(info, w, 21, 4.0)
    assert roof["achieved"] == pytest.approx(2e6 / 4e-3 / 1e9, rel=1e-12)
    assert roof["multiply_adds_per_launch"] == 21 * 2_000_000
    # two passes of 16 right-hand sides, three TF32 products per value and RHS
    assert roof["tf32_tensor_flops_per_launch"] == 2e6 * 16 * 2 * 3 * 2
    if sfu is None:
        assert roof["peak"] is None and roof["frac"] is None
    else:
        assert roof["peak"] == pytest.approx(152 * 16 * 2.07e9 / sfu / 1e9, rel=1e-12)
        assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"], rel=1e-12)


def test_column_relative_errors():
    ref = np.array([[3.0, 1.0], [4.0, 0.0]])
    f = ref + np.array([[0.0, 0.5], [0.5, 0.0]])
    e = bench._col_rel(f, ref)
    assert e["max"] == pytest.approx(0.5)
    assert e["median"] == pytest.approx((0.1 + 0.5) / 2)
    assert math.isfinite(e["max"])
