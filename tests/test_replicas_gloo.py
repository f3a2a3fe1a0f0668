"""The N>1 path of bench.py is independent replicas with no data-path collective; its
only cross-rank steps are the barrier and the max-over-ranks timing.  Checked here with
two gloo ranks on CPU (127.0.0.1 rendezvous)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r ran its replica in (10 + 5 r) ms moving 2e9 bytes per step
    ms, value = bench.replica_aggregate(10.0 + 5.0 * rank, 2e9, dist, device="cpu")
    dist.barrier()
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_replica_aggregate_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 15.0                          # slowest rank
        assert abs(value - 2 * 2e9 / 15e-3 / 1e9) < 1e-9   # all ranks' bytes / max time


def test_replica_aggregate_single_process():
    import bench
    ms, value = bench.replica_aggregate(20.0, 4e9)
    assert ms == 20.0 and abs(value - 200.0) < 1e-12
