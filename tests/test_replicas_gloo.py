"""Multi-process (replica) host logic of bench.py on CPU: world_size 2 over gloo.

The solver has no cross-GPU exchange; N > 1 runs independent replicas and the bench combines
them with a max over ranks of the time and a sum over ranks of the work.  These tests run that
combination with the gloo backend on the host.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    try:
        r, lr, w = bench.dist_env()
        assert (r, lr, w) == (rank, rank, world)
        bench.barrier(w)
        t_max = bench.reduce_max(10.0 + rank, w)       # slowest rank's time
        work = bench.reduce_sum(100.0 * (rank + 1), w)  # all ranks' work
        q.put((rank, t_max, work))
    finally:
        dist.destroy_process_group()


def test_replica_reductions_world2():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, t_max, work in got:
        assert t_max == 11.0
        assert work == 300.0


def test_single_process_reductions_are_identity():
    import bench
    assert bench.reduce_max(3.5, 1) == 3.5
    assert bench.reduce_sum(7.0, 1) == 7.0
    bench.barrier(1)
