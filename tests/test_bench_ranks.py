"""The bench's multi-rank aggregation (replicas, one per rank): max over ranks
of the step time, sum of the work units.  world_size 2 on the gloo backend,
CPU only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms, units = bench.combine_ranks(1.0 + rank, 100.0 * (rank + 1))
    out[rank] = (ms, units)
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_gloo_world2():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
    assert all(p.exitcode == 0 for p in procs)
    assert out[0] == (2.0, 300.0) and out[1] == (2.0, 300.0)


def test_combine_ranks_single_process_is_identity():
    import bench

    assert bench.combine_ranks(3.5, 42.0) == (3.5, 42.0)
