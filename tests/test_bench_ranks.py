"""Host-side logic of the multi-rank benchmark on CPU: two gloo ranks, each
with its own shard of data centers, combine their timings (maximum over
ranks) and counts (sum over ranks) the way the job-wide figures need."""
import os
import socket
import sys
import types

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        args = types.SimpleNamespace(instances=4, requests=2)
        wl = bench.workload(args, rank)
        hosts = sum(i.hosts for i in wl.instances)
        first = int(wl.instances[0].pre_cpu.sum())
        times, counts = bench.reduce_over_ranks(
            dist, [1.0 + rank, 10.0 * (1 - rank)], [rank + 1, 5, hosts], "cpu")
        empty_t, empty_c = bench.reduce_over_ranks(dist, [0.5 * rank], [], "cpu")
        out.put((rank, times, counts, hosts, first, empty_t, empty_c))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_times_sum_counts():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, t0, c0, h0, f0, e0, ec0), (_, t1, c1, h1, f1, e1, ec1) = res
    assert t0 == t1 == [2.0, 10.0]
    assert c0 == c1 == [3, 10, h0 + h1]
    assert e0 == e1 == [0.5] and ec0 == ec1 == []
    # weak scaling: same shape of work per rank, different data centers
    assert h0 == h1
    assert f0 != f1


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(None, [1.5, 2], [3, 4], "cpu") == ([1.5, 2.0], [3, 4])
