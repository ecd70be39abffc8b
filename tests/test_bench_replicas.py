"""The multi-GPU path of bench.py is replicas only (independent plans, no data
exchange).  Its whole-job accounting -- units of all ranks over the slowest
rank's time -- is checked here with world_size 2 gloo ranks on the CPU."""
import os

import pytest

torch = pytest.importorskip("torch")


def _rank(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    rate, ms, units = bench.replica_rate(10.0 * (rank + 1), 5 + rank, device="cpu")
    out[rank] = (rate, ms, units)
    dist.destroy_process_group()


def test_replica_rate_takes_slowest_rank_and_sums_units():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    port = 29500 + os.getpid() % 1000
    mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
    for r in range(2):
        rate, ms, units = out[r]
        assert ms == 20.0 and units == 11.0
        assert abs(rate - 11.0 / 0.020) < 1e-9


def test_replica_rate_single_process():
    import bench
    assert bench.replica_rate(4.0, 2) == (500.0, 4.0, 2)
