"""The N > 1 path of the bench (replicas, one process per GPU) on CPU: two gloo ranks reduce
their timings and pair counts exactly as the bench does (slowest rank's time, all ranks'
pairs)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, pairs = bench.reduce_over_ranks(dist, torch, torch.device("cpu"), 0.5 + rank, 1638 * (rank + 1))
    out[rank] = (t, pairs)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_reduction_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        assert dict(out) == {0: (1.5, 1638 * 3), 1: (1.5, 1638 * 3)}


def test_single_rank_is_identity():
    import torch
    import bench
    assert bench.reduce_over_ranks(None, torch, torch.device("cpu"), 0.25, 7) == (0.25, 7)
