"""The multi-GPU path of bench.py is replicas: every rank solves its own copy
of the workload and the only collectives are the timing barrier and the
max/sum of two scalars.  These run here as two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        # rank r took 10 (r + 1) ms and converged 32 - r solves
        ms, solves = bench.reduce_over_ranks(10.0 * (rank + 1), 32 - rank, "cpu")
        q.put((rank, ms, solves, solves / (ms / 1e3)))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_sum_the_solves():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs), [p.exitcode for p in procs]
    out = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, solves, value in out:
        assert ms == 20.0
        assert solves == 63.0
        assert value == pytest.approx(63.0 / 0.020)


def test_single_process_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert not dist.is_initialized()
    assert bench.reduce_over_ranks(12.5, 32, "cpu") == (12.5, 32.0)
