"""Host logic of the multi-GPU bench (replicas, weak scaling) on CPU: two
gloo ranks aggregate their timings with a max over ranks, and the whole-job
throughput counts every rank's simulations."""
import os
import socket

import pytest


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        elapsed = 100.0 + 25.0 * rank  # ms, a slower second rank
        mx = bench.max_over_ranks(elapsed, dist, "cpu")
        q.put((rank, mx, bench.job_throughput(512, 10, mx / 1000.0, world)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_and_count_all_simulations():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
    assert all(p.exitcode == 0 for p in procs)
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, mx, value in got:
        assert mx == 125.0
        assert value == pytest.approx(2 * 512 * 10 / 0.125)


def test_single_process_aggregation_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_throughput(512, 4, 2.0, 1) == 1024.0
