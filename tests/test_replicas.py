"""Multi-rank path (replicas): world_size-2 gloo processes on the CPU check
the reduction bench.py applies to its timed region (max time, summed work)."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_2501_08293_b300.replicas import aggregate
    t, n = aggregate(1.5 + rank, 1000 * (rank + 1), device="cpu")
    dist.barrier()
    q.put((rank, t, n))
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, n in out:
        assert t == 2.5 and n == 3000.0


def test_single_process_is_identity():
    from paper_2501_08293_b300.replicas import aggregate
    assert aggregate(2.0, 7) == (2.0, 7.0)
