"""Two-rank (gloo, CPU) check of the replica timing logic used by bench.py."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2108_13830_gb300 import replicas


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = replicas.rank_env()
    dist.barrier()
    elapsed = 100.0 + 50.0 * rank            # rank 1 is the slow one
    m = replicas.max_over_ranks(elapsed, dist)
    dist.barrier()
    q.put((r, w, lr, m, replicas.seed_offset(r)))
    dist.destroy_process_group()


def test_two_rank_max_and_throughput():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == 2 for o in out)
    assert all(o[3] == 150.0 for o in out)     # every rank sees the slowest time
    assert out[0][4] != out[1][4]              # replicas draw different inputs
    assert replicas.aggregate_throughput(4096, 2, 3, 150.0) == pytest.approx(2 * 4096 * 3 / 0.15)


def test_single_process_is_identity():
    assert replicas.max_over_ranks(12.5) == 12.5
