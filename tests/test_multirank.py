"""The N > 1 path of bench.py on CPU: ranks run independent replicas (images
do not interact, so there is no data exchange) and the job is timed by the
slowest rank.  world_size 2 over gloo, 127.0.0.1."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = bench._rank_env()
        local_ms = 100.0 + 50.0 * rank  # rank 1 is slower
        mx = bench.aggregate_max_ms(local_ms, w)
        rate = bench.job_throughput(1000, 4, w, mx)
        q.put((r, w, lr, mx, rate))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_time_by_the_slowest_rank():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1]
    for r, w, lr, mx, rate in res:
        assert w == 2 and lr == r
        assert mx == 150.0  # every rank sees the max
        assert rate == pytest.approx(2 * 1000 * 4 / 0.150)


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.aggregate_max_ms(12.5, 1) == 12.5
    assert bench.job_throughput(10, 2, 1, 1000.0) == 20.0
