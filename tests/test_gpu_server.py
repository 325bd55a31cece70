"""The serving runtime (rabitq_server_*): requests from several host threads,
batched per (index, k) into plan replays, results on the host equal a direct
search of the same queries; requests queued together run as one batch;
admission refuses what the device staging budget cannot hold.

eps0 = 6 makes a failed error bound practically impossible (Theorem 3.2), so
every result is the exact top-k of the probed buckets, whatever random
rounding a query's position in its batch draws."""
import threading

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

EPS = 6.0


@pytest.fixture(scope="module")
def R():
    import torch
    from paper_2405_12497_gb300 import build, rabitq
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    return rabitq


@pytest.fixture(scope="module")
def indices(R):
    from paper_2405_12497_gb300 import synth
    d1, q1 = synth.tiny(n=8000, nq=200)
    d2, q2 = synth.tiny(n=6000, d=200, nq=200)
    return [(R.Index.build(d1, 32, seed=2), q1), (R.Index.build(d2, 24, seed=2), q2)]


def test_server_results_equal_direct_search(R, indices):
    srv = R.Server(max_batch=128, mem_budget=8 << 20)
    slots = [srv.add_index(G, nprobe=6, eps0=EPS) for G, _ in indices]
    rng = np.random.default_rng(1)
    reqs = []
    for _ in range(60):
        i = int(rng.integers(0, 2))
        k = int(rng.choice([10, 20]))
        n = int(rng.integers(1, 41))
        o = int(rng.integers(0, 200 - n))
        reqs.append((i, k, o, n))
    outs = [None] * len(reqs)
    errs = []

    def client(part):
        try:
            for j in part:
                i, k, o, n = reqs[j]
                ids = np.zeros((n, k), np.int64)
                dist = np.zeros((n, k), np.float32)
                t = srv.submit(slots[i], indices[i][1][o:o + n], k, ids, dist)
                lat = srv.wait(t, 120.0)
                assert lat > 0
                outs[j] = (ids, dist)
        except Exception as e:  # noqa: BLE001 -- reported below
            errs.append(e)

    th = [threading.Thread(target=client, args=(list(range(c, len(reqs), 3)),)) for c in range(3)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    for (i, k, o, n), (ids, dist) in zip(reqs, outs):
        G, Q = indices[i]
        ri, rd = G.search(Q[o:o + n], k, 6, eps0=EPS)
        assert np.array_equal(ids, ri)
        assert np.array_equal(dist.view(np.uint32), rd.view(np.uint32))
    st = srv.stats()
    assert st["admitted"] == len(reqs) and st["refused"] == 0
    assert st["batched_requests"] == len(reqs) and st["in_flight_bytes"] == 0
    srv.free()


def test_server_batches_queued_requests(R, indices):
    """With a batching window, requests submitted back to back run together."""
    G, Q = indices[0]
    srv = R.Server(max_batch=256, mem_budget=8 << 20, batch_window_us=50_000)
    slot = srv.add_index(G, nprobe=6, eps0=EPS)
    bufs, tickets = [], []
    for j in range(8):
        ids = np.zeros((10, 10), np.int64)
        dist = np.zeros((10, 10), np.float32)
        tickets.append(srv.submit(slot, Q[10 * j:10 * j + 10], 10, ids, dist))
        bufs.append((ids, dist))
    for t in tickets:
        srv.wait(t, 60.0)
    st = srv.stats()
    assert st["batches"] < 8 and st["batched_queries"] == 80
    ri, _ = G.search(Q[:80], 10, 6, eps0=EPS)
    assert np.array_equal(np.concatenate([b[0] for b in bufs]), ri)
    srv.free()


def test_server_admission_by_device_budget(R, indices):
    G, Q = indices[0]
    srv = R.Server(max_batch=256, mem_budget=4096)          # room for 8 queries of d = 128
    slot = srv.add_index(G, nprobe=4, eps0=EPS)
    ids = np.zeros((40, 10), np.int64)
    dist = np.zeros((40, 10), np.float32)
    with pytest.raises(R.RabitqError) as e:
        srv.submit(slot, Q[:40], 10, ids, dist)
    assert e.value.code == R.EBUSY
    t = srv.submit(slot, Q[:8], 10, ids[:8], dist[:8])
    srv.wait(t, 60.0)
    st = srv.stats()
    assert st["refused"] == 1 and st["admitted"] == 1
    with pytest.raises(R.RabitqError):
        srv.submit(slot, Q[:4], 2000, ids, dist)             # k out of range
    srv.free()


def test_server_slots_added_while_serving(R, indices):
    """Indices added from one thread while three others submit and wait:
    the slot list grows under the server's lock and is read there; every
    result equals a direct search, and a slot added last serves too."""
    (G, Q), (G2, Q2) = indices
    srv = R.Server(max_batch=64, mem_budget=8 << 20)
    slot0 = srv.add_index(G, nprobe=6, eps0=EPS)
    errs, added, outs = [], [], []

    def adder():
        try:
            for _ in range(300):
                added.append(srv.add_index(G2, nprobe=4, eps0=EPS))
        except Exception as e:  # noqa: BLE001 -- reported below
            errs.append(e)

    def client(c):
        try:
            for j in range(20):
                o = (c * 20 + j) * 3 % 190
                ids = np.zeros((10, 10), np.int64)
                dist = np.zeros((10, 10), np.float32)
                srv.wait(srv.submit(slot0, Q[o:o + 10], 10, ids, dist), 120.0)
                outs.append((o, ids, dist))
        except Exception as e:  # noqa: BLE001 -- reported below
            errs.append(e)

    th = [threading.Thread(target=adder)] + [threading.Thread(target=client, args=(c,))
                                             for c in range(3)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    assert not errs, errs
    assert sorted(added) == list(range(1, 301)) and len(outs) == 60
    for o, ids, dist in outs:
        ri, rd = G.search(Q[o:o + 10], 10, 6, eps0=EPS)
        assert np.array_equal(ids, ri) and np.array_equal(dist.view(np.uint32), rd.view(np.uint32))
    ids = np.zeros((5, 10), np.int64)
    dist = np.zeros((5, 10), np.float32)
    srv.wait(srv.submit(added[-1], Q2[:5], 10, ids, dist), 120.0)
    ri, rd = G2.search(Q2[:5], 10, 4, eps0=EPS)
    assert np.array_equal(ids, ri) and np.array_equal(dist.view(np.uint32), rd.view(np.uint32))
    srv.free()
