"""The multi-rank path of bench.py (independent replicas, one per rank): whole-job
time is the slowest rank's, projections are summed over ranks.  Two gloo ranks on
the CPU, rendezvous on 127.0.0.1."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist          # noqa: E402
import torch.multiprocessing as mp        # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, u = bench.replica_totals(100.0 + 50.0 * rank, 1000 * (rank + 1), world, "cpu")
        out[rank] = (t, u)
    finally:
        dist.destroy_process_group()


def test_replica_totals_two_ranks():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        assert res[rank] == (150.0, 3000.0)


def test_replica_totals_single_rank():
    import bench
    assert bench.replica_totals(12.5, 7, 1, "cpu") == (12.5, 7.0)
