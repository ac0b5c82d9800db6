"""Host-side parts of the solve server: request streams, the served family, percentile
summaries, and option validation through the C ABI (no device work)."""
import math

import numpy as np
import pytest

from paper_2508_05958_gb300 import serving


def test_family_matches_the_served_mix():
    ops = serving.family()
    assert len(ops) == 9 + 18
    d2 = [o for o in ops if o.d == 2]
    assert {o.n for o in d2} == {256, 512, 1024} and {o.r for o in d2} == {5, 6, 7}
    assert all(o.leaf == 8 and abs(o.eta - math.sqrt(2)) < 1e-15 for o in d2)
    d3 = [o for o in ops if o.d == 3]
    assert {(o.n, o.leaf) for o in d3} == {(32, 4), (64, 8), (128, 8)}
    assert len(serving.family(max_n2=512, max_n3=64)) == 6 + 12


def test_a_is_in_natural_order():
    o = serving.OpSpec(3, 8, 1, 5, 4, 1.0, "sin")
    a = o.a().reshape(8, 8, 8)         # [i3, i2, i1]: dimension 1 fastest
    x1 = (np.arange(8) + 0.5) / 8
    assert np.allclose(a[3, 5, :], 1 + 0.5 * np.sin(2 * math.pi * x1))
    assert np.all(a == a[0:1, 0:1, :])


def test_poisson_stream_rate_and_determinism():
    t = serving.poisson_arrivals(200.0, 20000, seed=5)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1 / 200.0) < 3 * (1 / 200.0) / math.sqrt(20000)
    # exponential gaps: coefficient of variation 1
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.03
    s1 = serving.request_stream(serving.family(), 200.0, 50, seed=9)
    s2 = serving.request_stream(serving.family(), 200.0, 50, seed=9)
    assert s1 == s2 and len({i for _, i, _ in s1}) > 10
    assert all(b[0] > a[0] for a, b in zip(s1, s1[1:]))


def test_percentile_nearest_rank():
    xs = list(range(1, 101))
    assert serving.percentile(xs, 50) == 50 and serving.percentile(xs, 99) == 99
    assert serving.percentile([3.0], 99) == 3.0


@pytest.mark.parametrize("bad", [dict(max_active=0), dict(max_batch=0), dict(max_batch=65),
                                 dict(restart=0), dict(tol=0.0), dict(mixed=2),
                                 dict(inner_tol=1.5), dict(inner_precision=7),
                                 dict(autotune_ms=-1.0)])
def test_server_rejects_invalid_options(bad):
    import ctypes
    from paper_2508_05958_gb300 import htlr
    L = htlr.load()
    o = htlr.server_options(**bad)
    h = ctypes.c_void_p()
    assert L.htlr_server_create(ctypes.byref(o), ctypes.byref(h)) == htlr.HTLR_EINVAL
    assert h.value is None
    assert "invalid options" in htlr.htlr_last_error()
