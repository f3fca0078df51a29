"""bench.py's multi-rank logic on two CPU ranks over gloo: the barrier, the maximum over ranks of the
timed region and the whole-job value (the units every rank processed over the slowest rank's time).
The ranks are independent replicas; nothing else crosses between them."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q) -> None:
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        bench.barrier(w)
        total_ms = bench.reduce_max(w, 100.0 + 60.0 * r)  # rank 1 is the slow one
        q.put((r, w, local, total_ms, bench.job_value(w, 256, 20, total_ms)))
        bench.barrier(w)
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [g[:3] for g in got] == [(0, 2, 0), (1, 2, 1)]
    # every rank sees the maximum, and the value counts both ranks' requests over it
    assert all(g[3] == 160.0 for g in got)
    assert all(abs(g[4] - 2 * 256 * 20 / 0.160) < 1e-6 for g in got)


def test_one_rank_is_the_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(1, 12.5) == 12.5
    assert bench.job_value(1, 256, 20, 163.0) == 256 * 20 / 0.163
