"""Seeded request streams for the solve server and a driver that replays them.

The served family is the second-kind problem a(x) u + K u = f on uniform grids:
  d=2: n in {256, 512, 1024}, kernel log|x-y|, a = 1, leaf 8^2;
  d=3: n in {32, 64, 128}, kernel 1/|x-y| or exp(-|x-y|), a = 1 + 0.5 sin(2 pi x_1),
       leaf 4^3 for n=32 and 8^3 above;
with Chebyshev order r in {5, 6, 7} and eta = 1 (d=3) or sqrt(2) (d=2, non-adjacent).
Requests arrive as a Poisson process (exponential gaps, seeded); each draws its
operator uniformly from the family and f ~ N(0, 1) from a per-request seed.  The
bounded family (`max_n2`, `max_n3`) keeps a benchmark run to minutes.

This module only generates inputs and summarises timings; the solves run in the
library (htlr_server_*).
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass

import numpy as np

from .workloads import K_EXP_R, K_INV_R, K_LOG

STORE_SHARED = 2


@dataclass(frozen=True)
class OpSpec:
    d: int
    n: int
    ktype: int
    r: int
    leaf: int
    eta: float
    a_kind: str

    @property
    def N(self) -> int:
        return self.n ** self.d

    def a(self):
        """a(x) in natural order (dimension 1 fastest)."""
        if self.a_kind == "one":
            return np.ones(self.N)
        x1 = (np.arange(self.n) + 0.5) / self.n
        return np.tile(1.0 + 0.5 * np.sin(2 * math.pi * x1), self.N // self.n)

    def name(self) -> str:
        k = {K_LOG: "log", K_INV_R: "1/r", K_EXP_R: "exp(-r)"}[self.ktype]
        return f"d{self.d} n{self.n} {k} r{self.r}"


def family(max_n2: int = 1024, max_n3: int = 128):
    """The served operator family, optionally bounded in n."""
    ops = []
    for n in (256, 512, 1024):
        if n <= max_n2:
            for r in (5, 6, 7):
                ops.append(OpSpec(2, n, K_LOG, r, 8, math.sqrt(2.0), "one"))
    for n in (32, 64, 128):
        if n <= max_n3:
            for k in (K_INV_R, K_EXP_R):
                for r in (5, 6, 7):
                    ops.append(OpSpec(3, n, k, r, 4 if n == 32 else 8, 1.0, "sin"))
    return ops


def poisson_arrivals(rate: float, count: int, seed: int):
    """Arrival times (s) of `count` requests of a Poisson process of the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def request_stream(ops, rate: float, count: int, seed: int):
    """[(arrival_s, op_index, f_seed)] for `count` requests."""
    rng = np.random.default_rng(seed + 1)
    t = poisson_arrivals(rate, count, seed)
    which = rng.integers(0, len(ops), size=count)
    return [(float(t[i]), int(which[i]), int(seed * 100003 + i)) for i in range(count)]


def rhs(spec: OpSpec, f_seed: int):
    return np.random.default_rng(f_seed).standard_normal(spec.N)


def percentile(xs, q):
    """q-th percentile (0..100) by the nearest-rank rule."""
    xs = sorted(xs)
    if not xs:
        return float("nan")
    k = max(1, math.ceil(q / 100.0 * len(xs)))
    return xs[k - 1]


def replay(server, ops, stream, op_ids=None, keep_solutions=False):
    """Submit `stream` to a running htlr.Server at its arrival times (relative to now),
    wait for every request, and summarise.  Latency = completion - submission, on the
    server's clock."""
    if op_ids is None:
        op_ids = [server.add_operator(s.ktype, s.d, s.n, s.leaf, s.r, s.eta, a=s.a(),
                                      storage=STORE_SHARED) for s in ops]
    fs = [rhs(ops[i], seed) for (_, i, seed) in stream]
    t0 = time.perf_counter()
    ids = []
    for (t, i, _), f in zip(stream, fs):
        lag = t - (time.perf_counter() - t0)
        if lag > 0:
            time.sleep(lag)
        ids.append(server.submit(op_ids[i], f))
    results = [server.wait(r) for r in ids]
    wall = time.perf_counter() - t0
    infos = [inf for _, inf in results]
    lat = [inf["done_s"] - inf["submit_s"] for inf in infos]
    # service time: admission (a slot and memory granted) to completion; queueing: the
    # wait from submission to admission
    svc = [inf["done_s"] - inf["admit_s"] for inf in infos]
    queue = [inf["admit_s"] - inf["submit_s"] for inf in infos]
    first = min(inf["submit_s"] for inf in infos)
    last = max(inf["done_s"] for inf in infos)
    out = {
        "requests": len(ids),
        "completed": sum(inf["status"] == 2 for inf in infos),
        "converged": sum(bool(inf["converged"]) for inf in infos),
        "p50_ms": 1e3 * percentile(lat, 50),
        "p99_ms": 1e3 * percentile(lat, 99),
        "mean_ms": 1e3 * float(np.mean(lat)),
        "service_p50_ms": 1e3 * percentile(svc, 50),
        "service_p99_ms": 1e3 * percentile(svc, 99),
        "queue_p50_ms": 1e3 * percentile(queue, 50),
        "queue_p99_ms": 1e3 * percentile(queue, 99),
        "solves_per_s": len(ids) / (last - first),
        "makespan_s": last - first,
        "wall_s": wall,
        "max_rel_residual": max(inf["rel_residual"] for inf in infos),
        "iterations_mean": float(np.mean([inf["iterations"] for inf in infos])),
        "matvec_columns_mean": float(np.mean([inf["matvecs"] for inf in infos])),
    }
    if keep_solutions:
        out["solutions"] = [u for u, _ in results]
        out["infos"] = infos
    return out
