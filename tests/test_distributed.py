"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2): each rank
draws its own seeded batch (weak scaling, no collective on the data path) and
the timed region is reduced with MAX over ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2403_16665_gb300 import signals


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # each rank: its own batch (seed 2 + rank), as bench.py does
    x, _ = signals.batch_r32(batch=2, N=256, alpha=8, seed=2 + rank)
    digest = torch.tensor([float(np.float64(x.sum()))])
    allsum = [torch.zeros(1) for _ in range(world)]
    dist.all_gather(allsum, digest)
    # max over ranks of the per-rank time
    t = torch.tensor([1.0 + rank], dtype=torch.float64)
    dist.barrier()
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    q.put((rank, [float(v) for v in allsum], float(t.item())))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_host_logic():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    sums0, sums1 = res[0][1], res[1][1]
    assert sums0 == sums1                   # both ranks see the same gathered digests
    assert sums0[0] != sums0[1]             # and the two ranks' batches differ
    assert res[0][2] == res[1][2] == 2.0    # MAX over ranks
