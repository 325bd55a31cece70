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


# ------------------------------------------------------ bucket-sharded search
def _shard_worker(rank, world, port, out):
    """One rank = one shard: the oracle searches the shard's points (built
    with the global centroids and rotation), the ranks all-gather their
    (distance, id) top-k lists and every rank merges them."""
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as O
    from paper_2405_12497_gb300 import rabitq, synth
    data, Q = synth.tiny(n=6000, nq=60)
    K, k, nprobe = 24, 10, 6
    full = O.OracleIndex(data, K=K, seed=2, iters=6)
    shard_of, pts = rabitq.shard_clusters(np.diff(full.bucket_off), world)
    rows = np.flatnonzero(shard_of[full.assign] == rank)
    mine = O.OracleIndex(data[rows], K=K, seed=2, centroids=full.centroids)
    ids, dist_ = mine.search(Q, k, nprobe)
    gids = np.where(ids >= 0, rows[np.clip(ids, 0, None)], -1)
    t_ids = [torch.zeros_like(torch.from_numpy(gids)) for _ in range(world)]
    t_dist = [torch.zeros_like(torch.from_numpy(dist_)) for _ in range(world)]
    dist.all_gather(t_ids, torch.from_numpy(gids))
    dist.all_gather(t_dist, torch.from_numpy(dist_))
    all_i = np.concatenate([t.numpy() for t in t_ids], 1)
    all_d = np.concatenate([t.numpy() for t in t_dist], 1)
    merged = np.full((len(Q), k), -1, np.int64)
    for q in range(len(Q)):
        ok = all_i[q] >= 0
        order = np.lexsort((all_i[q][ok], all_d[q][ok]))[:k]
        merged[q, :len(order)] = all_i[q][ok][order]
    out.put((rank, merged, int(pts[rank]), len(rows)))
    dist.destroy_process_group()


def test_bucket_sharded_search_gloo():
    """Bucket sharding over two ranks (§4's buckets split by size): merged
    top-k lists equal the unsharded oracle search, query by query, except
    where a true neighbour's error bound failed."""
    import numpy as np
    import torch.multiprocessing as mp
    from oracle import oracle as O
    from paper_2405_12497_gb300 import build, synth
    build.build()
    O.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert np.array_equal(res[0][1], res[1][1])          # every rank merged the same
    assert res[0][2] == res[0][3] and res[1][2] == res[1][3]
    assert res[0][3] + res[1][3] == 6000
    assert abs(res[0][3] - res[1][3]) < 0.2 * 6000        # balanced shards
    data, Q = synth.tiny(n=6000, nq=60)
    full = O.OracleIndex(data, K=24, seed=2, iters=6)
    ids, _ = full.search(Q, 10, 6)
    merged = res[0][1]
    for qi in range(len(Q)):
        if np.array_equal(merged[qi], ids[qi]):
            continue
        # a mismatch must come from a failed bound of a true neighbour
        t = full.trace(Q[qi], qi, 10, 6)
        ex = O.sqdist_matrix(Q[qi:qi + 1], full.data[t["pair_id"]])[0]
        failed = (t["pair_est"][:, 1] > ex) | (t["pair_est"][:, 2] < ex)
        assert failed.any(), qi
