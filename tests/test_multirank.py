"""The multi-rank harness of bench.py on CPU (gloo, world size 2): queries
are independent, so ranks run replicas of the search with no collective on
the data path; the only collectives are the timed region's barrier and the
max-reduction that makes the job's time its slowest rank's.
"""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # each rank's "timed region" differs; the job's time is the largest
    t = bench.max_over_ranks(10.0 + 7.5 * rank, dist, "cpu")
    dist.barrier()
    rate = bench.job_rate(world, 10_000, t / 1e3)
    out.put((rank, t, rate))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    assert all(t == 17.5 for _, t, _ in res)              # the slower rank's time
    assert all(rate == pytest.approx(2 * 10_000 / 0.0175) for _, _, rate in res)


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25
    assert bench.job_rate(1, 100, 0.5) == 200.0
