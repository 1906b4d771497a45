"""Multi-GPU runs are replicas (the method here does not shard): every rank simulates
its own circuit and the job reports all ranks' work over the slowest rank's time.  The
host-side reduction is checked with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms, upd = bench.reduce_over_ranks(10.0 + 5.0 * rank, 1000.0 * (rank + 1), dist, "cpu")
    out[rank] = (ms, upd, bench.replica_seed(rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_the_bench():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    for r in (0, 1):
        ms, upd, _ = res[r]
        assert ms == 15.0  # the slowest rank's time
        assert upd == 3000.0  # all ranks' amplitude updates
    assert res[0][2] != res[1][2]  # independent circuits


def test_replica_circuits_differ_per_rank():
    import bench
    from paper_1911_04034_gb300 import circuits as Cc

    a = Cc.rcs(2, 3, 4, seed=bench.replica_seed(0))
    b = Cc.rcs(2, 3, 4, seed=bench.replica_seed(1))
    assert len(a) == len(b) and (a["u"] != b["u"]).any()
