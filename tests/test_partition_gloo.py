"""Host side of the T-partitioned operator on CPU: the face routing of
partition.TorchFaceExchange between 2 and 4 gloo ranks (each rank's first-timeslice face
reaches the rank below as its upper halo, its last-timeslice face the rank above as its
lower halo, periodically), and the splitting of links and fields into partitions."""
import os
import socket

import numpy as np
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
    from paper_1810_01609_gb300.partition import TorchFaceExchange
    x = TorchFaceExchange(64, device="cpu")
    x.send_lo.fill_(2 * rank + 1)     # first timeslice of rank r
    x.send_hi.fill_(2 * rank + 2)     # last timeslice of rank r
    x.exchange()
    q.put((rank, int(x.recv_lo[0]), int(x.recv_hi[0]), bool((x.recv_lo == x.recv_lo[0]).all()),
           bool((x.recv_hi == x.recv_hi[0]).all())))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 4])
def test_face_routing_gloo(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, lo, hi, lo_ok, hi_ok in res:
        assert lo_ok and hi_ok
        assert lo == 2 * ((rank - 1) % world) + 2      # the lower rank's last timeslice
        assert hi == 2 * ((rank + 1) % world) + 1      # the upper rank's first timeslice


def test_split_links_and_fields():
    from paper_1810_01609_gb300.partition import split_links, split_t, join_t
    T = 8
    U = np.arange(T * 2 * 2 * 2 * 4 * 9, dtype=np.float64).reshape(T, 2, 2, 2, 4, 3, 3)
    parts = split_links(U, 4)
    for r, u in enumerate(parts):
        assert u.shape[0] == 3
        assert np.array_equal(u[0], U[(2 * r - 1) % T])      # ghost: the lower neighbour's last slice
        assert np.array_equal(u[1:], U[2 * r:2 * r + 2])
    f = np.arange(2 * 3 * T * 4).reshape(2, 3, T, 4)
    assert np.array_equal(join_t(split_t(f, 4, 2), 2), f)
