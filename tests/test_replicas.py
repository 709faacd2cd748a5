"""The multi-rank path of bench.py (N replicas, no collective on the data path) on CPU with gloo,
world size 2: the whole-job value is all ranks' transforms over the slowest rank's time, every rank
agrees on it, and the reference arm runs on rank 0 only."""
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


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank r "took" 10 (r + 1) ms for 5 steps of 256 transforms
    value, ms_max = bench.replica_value(256, world, 5, 10.0 * (rank + 1))
    bench.barrier(world)

    class A:
        steps = 1
        warmup = 0

    ref_rc = bench.run_reference(A) if rank != 0 else None  # rank != 0 leaves at once, without work
    q.put((rank, value, ms_max, ref_rc))
    dist.destroy_process_group()


def test_replica_value_and_rank_roles_under_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    ms_slowest = 10.0 * world
    want = 256 * world * 5 / (ms_slowest / 1000.0)
    for rank, value, ms_max, ref_rc in res:
        assert ms_max == ms_slowest
        assert value == pytest.approx(want)
    assert res[1][3] == 0  # the reference arm on rank 1 exits 0 without running the oracle
