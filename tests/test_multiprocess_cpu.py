"""The multi-process (replicas) path on CPU: two gloo ranks, no GPU.

The smoother shards by image with no data-path collective; the only cross-rank step is the
benchmark's timing aggregation (max over ranks) and the whole-job throughput formula.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        slowest = bench.max_over_ranks(10.0 + rank)          # rank 1 is the slow one
        q.put((rank, slowest, bench.replica_throughput(8.2944, slowest / 1e3, world)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [11.0, 11.0]
    for _, slowest, thr in got:
        assert thr == pytest.approx(2 * 8.2944 / 0.011)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_throughput(2.0, 0.5, 1) == 4.0
