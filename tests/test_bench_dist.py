"""The multi-rank bookkeeping of bench.py on CPU: two gloo ranks with different
step times agree on the slowest one, and the whole-job value counts every
rank's right-hand sides once (replicas, weak scaling)."""
import os

import pytest
import torch.multiprocessing as mp


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = 100.0 + 50.0 * rank          # rank 1 is slower
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        q.put((rank, ms, bench.job_value(world, 8, ms / 1e3)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 150.0
        assert value == pytest.approx(2 * 8 / 0.150)


def test_single_process_values():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_value(1, 8, 4.0) == 2.0
