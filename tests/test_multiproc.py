"""The benchmark's multi-rank host logic on CPU: two gloo ranks (replicas).

Every rank filters its own frames (no data-path collective); the barrier and
the max-over-ranks time are the only communication, and the whole-job rate
counts every rank's pixels over the slowest rank's time.
"""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench.dist_env()
    dist.barrier()
    elapsed = [12.0, 20.0][rank]                 # rank 1 is the slow replica
    mx = bench.reduce_max(elapsed, ws)
    rate = bench.whole_job_rate(1920 * 1080, ws, mx)
    q.put((r, ws, local, mx, rate, bench.frame_seed(r)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert all(r[3] == 20.0 for r in res)                       # max over ranks
    assert all(abs(r[4] - 2 * 1920 * 1080 / 0.020 / 1e6) < 1e-6 for r in res)
    assert res[0][5] != res[1][5]                               # replicas filter different frames
