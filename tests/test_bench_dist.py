"""The bench's multi-rank path on CPU (gloo, world size 2): every rank runs
an independent replica, the job's time is the slowest rank's and the value
counts all ranks' units; no collective touches the data path."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench._dist()
        bench._barrier(w)
        slowest = bench._max_over_ranks(w, 100.0 + 50.0 * r)  # rank 1 is slower
        q.put((r, w, slowest, bench.replica_throughput(w, 1e9, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_on_gloo():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, slowest, value in out:
        assert w == 2 and slowest == 150.0
        assert value == pytest.approx(2 * 1e9 / 0.150)


def test_replica_throughput_single_rank():
    import bench
    assert bench.replica_throughput(1, 5e9, 1000.0) == pytest.approx(5e9)
