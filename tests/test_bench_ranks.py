"""Host logic of the multi-rank benchmark on CPU (gloo, world size 2): the
ranks' right-hand sides are disjoint, and the timing reduction is the max."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    cols = bench.rank_columns(16384, 64, rank)
    t = torch.from_numpy(cols.astype("int64"))
    out = [torch.zeros_like(t) for _ in range(world)]
    dist.all_gather(out, t)
    mx = bench.reduce_max(1.0 + rank, world, "cpu")
    if rank == 0:
        q.put(([o.tolist() for o in out], mx))
    dist.barrier()
    dist.destroy_process_group()


def test_rank_split_and_max_over_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    cols, mx = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert len(cols[0]) == 64 and len(cols[1]) == 64
    assert not set(cols[0]) & set(cols[1])
    assert mx == 2.0
