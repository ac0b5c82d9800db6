"""Seeded synthetic workloads: grids, a(x) and right-hand sides.

This module only generates inputs; it holds none of the HTLR arithmetic.  Both the CUDA
path and the CPU oracle take their inputs from here.  The shapes follow the paper's
experiments (uniform grids on [0,1]^d, random vectors; §5) and the four workload
configurations this library is measured on:

  c1  d=2, n=64 (N=4096),   log|x-y|,    a=1,                       leaf 8^2, p=6, non-adjacent (eta=sqrt 2), 1 RHS ~ U[-1,1]
  c2  d=3, n=32 (N=32768),  1/|x-y|,     a=1+0.5 sin(2 pi x_1),     leaf 4^3, p=5, eta=1,                     1 RHS ~ N(0,1)
  c3  d=3, n=128 (N=2^21),  1/|x-y|,     a=0,                       leaf 8^3, p=6, eta=1,                     64 RHS ~ N(0,1)
  c4  d=3, n=128 tensor quasi-uniform,   exp(-|x-y|), a=0,          leaf ~8^3, p=7, eta=1,                    16 RHS ~ N(0,1)

Random numbers come from numpy's PCG64 generator seeded per workload.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Kernel ids of the public C enum (include/htlr.h).
K_LOG, K_INV_R, K_EXP_R, K_GAUSS, K_POLY, K_CONST = range(6)


@dataclass
class Workload:
    name: str
    d: int
    n: int
    ktype: int
    leaf: int
    p: int
    eta: float
    nrhs: int = 1
    kscale: float = 1.0
    kparam: float = 0.0
    a_kind: str = "zero"          # "zero" | "one" | "sin"
    u_kind: str = "normal"        # "normal" | "uniform"
    grid_kind: str = "uniform"    # "uniform" | "quasi"
    seed: int = 1
    grid_seed: int = 101
    q: int = 16
    extra: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return self.n ** self.d

    # -- grid ---------------------------------------------------------------------
    def grid(self):
        """None for the uniform grid x_i = (i + 1/2)/n with cells [i/n, (i+1)/n];
        for the quasi-uniform tensor grid, a pair (x, edges) of shapes (d, n), (d, n+1)."""
        if self.grid_kind == "uniform":
            return None
        return quasi_uniform_tensor_grid(self.d, self.n, self.grid_seed)

    def coords(self):
        """Per-dimension grid-line coordinates, shape (d, n)."""
        g = self.grid()
        if g is None:
            x = (np.arange(self.n) + 0.5) / self.n
            return np.tile(x, (self.d, 1))
        return g[0]

    # -- a(x) ---------------------------------------------------------------------
    def a(self):
        """a(x_i) in natural order (first index fastest), or None for a = 0."""
        if self.a_kind == "zero":
            return None
        if self.a_kind == "one":
            return np.ones(self.N)
        if self.a_kind == "sin":
            x1 = self.coords()[0]
            idx = np.arange(self.N) % self.n
            return 1.0 + 0.5 * np.sin(2.0 * math.pi * x1[idx])
        raise ValueError(self.a_kind)

    # -- right-hand sides ---------------------------------------------------------
    def u(self, nrhs: int | None = None, seed: int | None = None):
        """N x nrhs column-major (Fortran-ordered) matrix of right-hand sides."""
        nrhs = self.nrhs if nrhs is None else nrhs
        rng = np.random.default_rng(self.seed if seed is None else seed)
        if self.u_kind == "uniform":
            U = rng.uniform(-1.0, 1.0, size=(nrhs, self.N)).T
        else:
            U = rng.standard_normal(size=(nrhs, self.N)).T
        return np.asfortranarray(U)

    def sample_rows(self, count: int, seed: int = 7):
        rng = np.random.default_rng(seed)
        return np.sort(rng.choice(self.N, size=min(count, self.N), replace=False)).astype(np.int64)


def quasi_uniform_tensor_grid(d: int, n: int, seed: int):
    """Quasi-uniform tensor grid: x = g(xi) + delta per coordinate line, with
    g(xi) = xi + 0.08 sin(2 pi xi)/(2 pi) on the uniform xi = (i+1/2)/n and one seeded
    jitter delta ~ U[-0.1 h, 0.1 h] per grid line (the grid stays a tensor grid).
    Cells are the 1-D Voronoi cells (midpoints; the end cells reach 0 and 1)."""
    rng = np.random.default_rng(seed)
    h = 1.0 / n
    xi = (np.arange(n) + 0.5) * h
    g = xi + 0.08 * np.sin(2.0 * math.pi * xi) / (2.0 * math.pi)
    xs = np.empty((d, n))
    es = np.empty((d, n + 1))
    for l in range(d):
        x = g + rng.uniform(-0.1 * h, 0.1 * h, size=n)
        xs[l] = x
        es[l, 0] = 0.0
        es[l, n] = 1.0
        es[l, 1:n] = 0.5 * (x[:-1] + x[1:])
    return xs, es


CONFIGS = {
    "c1": Workload("c1", d=2, n=64, ktype=K_LOG, leaf=8, p=6, eta=math.sqrt(2.0), nrhs=1,
                   a_kind="one", u_kind="uniform", seed=1),
    "c2": Workload("c2", d=3, n=32, ktype=K_INV_R, leaf=4, p=5, eta=1.0, nrhs=1,
                   a_kind="sin", u_kind="normal", seed=2),
    "c3": Workload("c3", d=3, n=128, ktype=K_INV_R, leaf=8, p=6, eta=1.0, nrhs=64,
                   a_kind="zero", u_kind="normal", seed=3),
    # the c2 grid under weak admissibility: the same block shapes (125 x 125 cores at
    # level 2, 64 x 64 at the leaves) but ~0.2 GB of blocks: the profiling case
    "c2_weak": Workload("c2_weak", d=3, n=32, ktype=K_INV_R, leaf=4, p=5, eta=0.0, nrhs=1,
                        a_kind="sin", u_kind="normal", seed=2),
    "c4": Workload("c4", d=3, n=128, ktype=K_EXP_R, leaf=8, p=7, eta=1.0, nrhs=16,
                   a_kind="zero", u_kind="normal", grid_kind="quasi", seed=4),
    # the c3 operator one level shallower (N = 262144, 64 RHS): the same core and near
    # block shapes (216 x 216, 512 x 512) with ~0.3 GB of vectors, for profiling captures
    "c3_n64": Workload("c3_n64", d=3, n=64, ktype=K_INV_R, leaf=8, p=6, eta=1.0, nrhs=64,
                       a_kind="zero", u_kind="normal", seed=3),
    # the c4 operator one level shallower (N = 262144, 16 RHS, quasi-uniform tensor grid):
    # the same 343-row cores and 7-9 point leaves, for profiling captures
    "c4_n64": Workload("c4_n64", d=3, n=64, ktype=K_EXP_R, leaf=8, p=7, eta=1.0, nrhs=16,
                       a_kind="zero", u_kind="normal", grid_kind="quasi", seed=4),
}


def workload(name: str, **over) -> Workload:
    """A named configuration, optionally with fields replaced (e.g. n=16 for tests)."""
    base = CONFIGS[name]
    kw = dict(base.__dict__)
    kw.update(over)
    return Workload(**kw)
