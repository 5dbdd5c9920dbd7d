"""Host logic of the multi-GPU form: independent replicas.

One solve does not shard (every smoother sweep and dot product would need an
exchange), so N GPUs run N independent solves; the ranks exchange only the
timing scalars, and rank 0 reports the maximum over ranks.  These tests run
that host logic as world-size-2 gloo process groups on the CPU.
"""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local = [10.0 + rank, 20.0 - rank, 3.0 * (rank + 1)]
    got = bench.max_over_ranks(local)
    ws, r, lr = bench.dist_env()
    out.put((rank, got, ws, r, lr, bench.replica_throughput(ws, got[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, ws, r, lr, thr in res:
        assert got == [11.0, 20.0, 6.0]
        assert ws == 2 and r == rank and lr == rank
        assert thr == pytest.approx(2 * 1e3 / 11.0)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks([1.5, 2.5]) == [1.5, 2.5]
    assert bench.replica_throughput(1, 8.0) == 125.0
