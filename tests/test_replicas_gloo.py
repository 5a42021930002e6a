"""The multi-rank bench path on CPU: two gloo ranks take the slowest rank's time and report
the whole job's throughput; each rank gets its own replica seed."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_seconds = 1.0 + rank  # rank 1 is the slow one
    t = bench.max_over_ranks(local_seconds, world)
    v = bench.aggregate_mlups(1_000_000, 10, t, world)
    out[rank] = (t, v, bench.replica_seed(5, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(2, port, out), nprocs=2, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 2.0          # max over ranks
    assert res[0][1] == res[1][1] == pytest.approx(2 * 1_000_000 * 10 / 2.0 / 1e6)
    assert {res[0][2], res[1][2]} == {5, 6}       # distinct replicas
