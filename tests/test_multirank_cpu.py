"""Replica (k-point-parallel) bench logic across ranks, on CPU with gloo.

k-points are independent, so N GPUs run N replicas with no collective on the
data path; the only cross-rank step is the max of the timed region over ranks
(and the barriers around it).  World size 2, 127.0.0.1 rendezvous.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, root, q):
    import sys
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench._dist()
    dist.barrier()
    t = bench.reduce_max(10.0 + 5.0 * rank, torch.device("cpu"))  # per-rank "ms"
    dist.barrier()
    q.put((rank, ws, r, local, t))
    dist.destroy_process_group()


def test_max_over_ranks_gloo(root):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, root, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [o[0] for o in out] == [0, 1]
    assert all(o[1] == 2 and o[2] == o[0] and o[3] == o[0] for o in out)
    assert all(o[4] == 15.0 for o in out)  # both ranks see the slowest rank's time


def test_reduce_max_without_process_group():
    import bench
    assert bench.reduce_max(3.5, torch.device("cpu")) == 3.5
