"""The N > 1 path of the benchmark on CPU: two `gloo` ranks run the replica aggregation
(max over ranks of the step time, summed throughput) and the reference arm's rank
handling.  The path shards by replicas only, so there is no data-path collective."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = bench.dist_env()
        ms = bench.max_over_ranks(1.5 + rank, w, "cpu")      # rank 1 is the slow one
        value = bench.replica_throughput(w, 32768, 1, ms)
        q.put((r, w, local, ms, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_benchmark():
    import multiprocessing as mp
    pytest.importorskip("torch")
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    for r, (rank, world, local, ms, value) in enumerate(got):
        assert (rank, world, local) == (r, 2, r)
        assert ms == 2.5                          # max over the two ranks
        assert abs(value - 2 * 32768 / 2.5e-3 / 1e9) < 1e-12


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.0, 1, "cpu") == 3.0
    assert bench.replica_throughput(1, 1000, 4, 2.0) == 1000 * 4 / 2e-3 / 1e9
