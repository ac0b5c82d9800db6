"""The seeded input recipe on the host: the quasi-uniform tensor grid keeps the properties
the readings of the paper rely on (a tensor grid, monotone lines, bounded jitter, 1-D
Voronoi cells, 7-9 points per leaf line at n = 128 with 16 leaves per dimension), and the
workloads are reproducible."""
import math

import numpy as np

from paper_2508_05958_gb300.workloads import quasi_uniform_tensor_grid, workload


def test_quasi_uniform_grid_properties():
    d, n = 3, 128
    h = 1.0 / n
    x, e = quasi_uniform_tensor_grid(d, n, seed=101)
    assert x.shape == (d, n) and e.shape == (d, n + 1)
    xi = (np.arange(n) + 0.5) * h
    g = xi + 0.08 * np.sin(2 * math.pi * xi) / (2 * math.pi)
    for l in range(d):
        assert np.all(np.abs(x[l] - g) <= 0.1 * h + 1e-15)       # one jitter per line
        assert np.all(np.diff(x[l]) > 0)                          # monotone
        assert e[l, 0] == 0.0 and e[l, n] == 1.0
        assert np.allclose(e[l, 1:n], 0.5 * (x[l, :-1] + x[l, 1:]), rtol=0, atol=0)
        assert np.all((x[l] > e[l, :-1]) & (x[l] < e[l, 1:]))     # each point in its cell
        # points per geometric leaf cell [k/16, (k+1)/16): 7 to 9
        counts = np.bincount(np.minimum((x[l] * 16).astype(int), 15), minlength=16)
        assert counts.min() >= 7 and counts.max() <= 9 and counts.sum() == n
        assert math.isclose(np.diff(e[l]).sum(), 1.0, rel_tol=1e-14)   # cells tile [0, 1]


def test_workloads_are_seeded_and_shaped():
    w = workload("c2")
    u1, u2 = w.u(), w.u()
    assert u1.shape == (w.N, 1) and u1.flags.f_contiguous and np.array_equal(u1, u2)
    a = w.a()
    assert a.shape == (w.N,) and np.all((a >= 0.5) & (a <= 1.5))
    c4 = workload("c4")
    g1, g2 = c4.grid(), c4.grid()
    assert np.array_equal(g1[0], g2[0]) and np.array_equal(g1[1], g2[1])
    assert c4.u(nrhs=2).shape == (c4.N, 2)
    rows = c4.sample_rows(1024, seed=1024)
    assert len(np.unique(rows)) == 1024 and rows.min() >= 0 and rows.max() < c4.N
