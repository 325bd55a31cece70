"""Parity of the inner-product / cosine metrics and of the single-code
estimator (CUDA path through the C-ABI) with the CPU oracle.

Bit-exact, as for the squared distance: k-means, codes and factors (the
inner-product factors of the closing footnote of §6), probe lists ranked by
-<q, c>, per-pair estimates and bounds, thresholds, survivor sets and the
final top-k with exact inner products; the single-code estimator's values
for any ids, on every scan path and launch form (plans, split batches,
tensor-core scan, the allocation-free entry point).
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    from paper_2405_12497_gb300 import build, rabitq
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    build.build()
    return rabitq


@pytest.fixture(scope="module", params=["ip", "cosine"])
def pair(request, R, oracle_mod, tiny_workload):
    data, _ = tiny_workload
    m = request.param
    G = R.Index.build(data, 16, seed=2, kmeans_iters=10, metric=m)
    O = oracle_mod.OracleIndex(data, K=16, seed=2, iters=10, metric=m)
    return m, G, O


def _same(a, b):
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(np.asarray(a[1]).view(np.uint32), np.asarray(b[1]).view(np.uint32))


def test_build_bit_exact(pair):
    m, G, O = pair
    assert G.metric == m
    assert np.array_equal(G.centroids().view(np.uint32), O.centroids.view(np.uint32))
    assert np.array_equal(G.assign(), O.assign)
    assert np.array_equal(G.codes(), O.codes)
    assert np.array_equal(G.factors().view(np.uint32), O.factors.view(np.uint32))


@pytest.mark.parametrize("k,nprobe,bq,eps0", [(10, 4, 4, 1.9), (100, 16, 4, 1.9), (1, 1, 1, 0.0),
                                               (25, 3, 8, 3.0)])
def test_search_bit_exact(pair, tiny_workload, k, nprobe, bq, eps0):
    import torch
    _, G, O = pair
    _, Q = tiny_workload
    ref = O.search(Q, k, nprobe, bq=bq, eps0=eps0)
    _same(G.search(Q, k, nprobe, bq=bq, eps0=eps0), ref)
    ids, dist = G.search(torch.from_numpy(Q).cuda(), k, nprobe, bq=bq, eps0=eps0)
    _same((ids.cpu().numpy(), dist.cpu().numpy()), ref)
    assert np.all(np.diff(ref[1], axis=1)[ref[0][:, 1:] >= 0] <= 0)  # descending values


def test_trace_bit_exact(R, pair, tiny_workload):
    """Per-pair estimates, thresholds and survivor sets equal the oracle's
    (scores -<o, q>; the probe list holds -<q, c>)."""
    import torch
    _, G, O = pair
    _, Q = tiny_workload
    t = R.Index.search_trace(G, torch.from_numpy(Q).cuda(), 10, 6, pair_cap=12000,
                             surv_cap=12000)
    for i in (0, 7, 55):
        o = O.trace(Q[i], i, 10, 6)
        assert np.array_equal(t["probe_ids"][i].cpu().numpy(), o["probe_ids"])
        assert np.array_equal(t["probe_dist"][i].cpu().numpy().view(np.uint32),
                              o["probe_dist"].view(np.uint32))
        assert np.array_equal(t["meta"][i].cpu().numpy().view(np.uint32),
                              o["meta"][:, :4].view(np.uint32))
        n = int(t["n_pairs"][i])
        assert np.array_equal(t["pair_id"][i, :n].cpu().numpy(), o["pair_id"])
        assert np.array_equal(t["pair_est"][i, :n].cpu().numpy().view(np.uint32),
                              o["pair_est"].view(np.uint32))
        for key in ("tau", "tau_ub", "tau1"):
            assert np.float32(t[key][i].item()).view(np.uint32) == \
                np.float32(o[key]).view(np.uint32), key
        ns = int(t["n_surv"][i])
        assert np.array_equal(np.sort(t["surv_ids"][i, :ns].cpu().numpy()), o["surv_ids"])


def test_padding_and_full_probe(pair, tiny_workload):
    _, G, O = pair
    _, Q = tiny_workload
    ids, ip = G.search(Q[:20], 1000, 1)
    _same((ids, ip), O.search(Q[:20], 1000, 1))
    assert (ids == -1).any() and np.all(ip[ids == -1] == -np.inf)
    _same(G.search(Q[:20], 10, 16), O.search(Q[:20], 10, 16))


def test_other_launch_forms_equal_search(R, pair, tiny_workload):
    """Plans (CUDA graphs), split small batches, the tensor-core scan and
    per-query probe counts give the same results."""
    import torch
    _, G, O = pair
    _, Q = tiny_workload
    big = np.concatenate([Q] * 6)
    ref = G.search(big, 10, 8, scan_path=R.SCAN_POPC)
    for nq in (1, 3, 50):                                          # split mode
        _same(G.search(Q[:nq], 10, 8, scan_path=R.SCAN_POPC), (ref[0][:nq], ref[1][:nq]))
    plan = R.Plan(G, 10, 8, 64)
    for nq in (1, 64):
        _same(plan.search(Q[:nq]), (ref[0][:nq], ref[1][:nq]))
    _same(G.search(Q, 10, 8, scan_path=R.SCAN_TC), (ref[0][:100], ref[1][:100]))
    npq = (np.arange(100) % 8 + 1).astype(np.int32)
    a = G.search(Q, 10, 8, per_query_nprobe=npq)
    for i in (0, 5, 99):  # query i's quantization stream is its index in the batch
        t = O.trace(Q[i], i, 10, int(npq[i]))
        _same((a[0][i], a[1][i]), (t["ids"], t["dist"]))
    # the allocation-free entry point
    qd = torch.from_numpy(Q).cuda()
    ids = torch.empty((100, 10), dtype=torch.int64, device="cuda")
    dist = torch.empty((100, 10), dtype=torch.float32, device="cuda")
    o = R.SearchOpts()
    R.lib().rabitq_search_opts_default(C.byref(o))
    o.io_on_device = 1
    o.stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = R.lib().rabitq_search_noalloc(G._h, C.c_void_p(qd.data_ptr()), 100, 10, 8, 4, 1.9,
                                       C.c_void_p(ids.data_ptr()), C.c_void_p(dist.data_ptr()),
                                       C.byref(o))
    torch.cuda.synchronize()
    assert rc == R.OK
    _same((ids.cpu().numpy(), dist.cpu().numpy()), (ref[0][:100], ref[1][:100]))


@pytest.mark.parametrize("n,d,K,nq", [(20_011, 100, 37, 300), (3001, 33, 40, 64)])
def test_ragged_inner_product_bit_exact(R, oracle_mod, n, d, K, nq):
    """Sizes that span several tiles, a dimension with no 16-byte rows and a
    ragged tail; a query equal to a data point and duplicate points."""
    rng = np.random.default_rng(n)
    data = (rng.standard_normal((n, d)) * rng.uniform(0.1, 3, d)).astype(np.float32)
    data[5] = data[6]
    Q = (rng.standard_normal((nq, d)) * 2).astype(np.float32)
    Q[3] = data[11]
    G = R.Index.build(data, K, seed=5, kmeans_iters=4, metric="ip")
    O = oracle_mod.OracleIndex(data, K=K, seed=5, iters=4, metric="ip", threads=8)
    assert np.array_equal(G.factors().view(np.uint32), O.factors.view(np.uint32))
    _same(G.search(Q, 20, 6), O.search(Q, 20, 6, threads=8))


def test_estimate_bit_exact(R, oracle_mod, tiny_workload, pair):
    """Single-code estimates for scattered ids (-1 slots give NaNs) equal the
    oracle's, for every metric, on host and device buffers."""
    import torch
    data, Q = tiny_workload
    rng = np.random.default_rng(3)
    ids = rng.integers(0, len(data), (100, 33)).astype(np.int64)
    ids[4, 7] = -1
    ids[9, :] = -1
    _, G, O = pair
    GL = R.Index.build(data, 16, seed=2, kmeans_iters=10)
    OL = oracle_mod.OracleIndex(data, K=16, seed=2, iters=10)
    for g, o in ((G, O), (GL, OL)):
        for bq, eps0 in ((4, 1.9), (1, 0.0), (8, 3.0)):
            want = o.estimate(Q, ids, bq=bq, eps0=eps0)
            got = g.estimate(Q, ids, bq=bq, eps0=eps0)
            assert np.array_equal(np.isnan(got), np.isnan(want))
            assert np.array_equal(got.view(np.uint32), want.view(np.uint32))
        got_d = g.estimate(torch.from_numpy(Q).cuda(), torch.from_numpy(ids).cuda())
        assert np.array_equal(got_d.cpu().numpy().view(np.uint32),
                              o.estimate(Q, ids).view(np.uint32))


def test_estimate_equals_scan_values(R, tiny_workload):
    """The estimates of the codes a search scanned equal the scan's own
    per-pair values (same quantization stream)."""
    import torch
    data, Q = tiny_workload
    G = R.Index.build(data, 16, seed=2, kmeans_iters=10, metric="ip")
    t = R.Index.search_trace(G, torch.from_numpy(Q[:8]).cuda(), 10, 5, pair_cap=12000)
    n = int(t["n_pairs"][6])
    ids = -np.ones((8, n), np.int64)
    ids[6] = t["pair_id"][6, :n].cpu().numpy()
    est = G.estimate(Q[:8], ids)
    pe = t["pair_est"][6, :n].cpu().numpy()
    assert np.array_equal(est[6].view(np.uint32), (-pe[:, [0, 2, 1]]).view(np.uint32))


def test_estimate_errors(R, tiny_workload):
    data, Q = tiny_workload
    G = R.Index.build(data, 16, seed=2, kmeans_iters=3)
    ids = np.zeros((2, 3), np.int64)
    ids[1, 2] = len(data)
    with pytest.raises(R.RabitqError) as e:
        G.estimate(Q[:2], ids)
    assert e.value.code == R.EINVAL
    ids[1, 2] = -5
    with pytest.raises(R.RabitqError):
        G.estimate(Q[:2], ids)
    with pytest.raises(R.RabitqError):
        G.estimate(Q[:2], np.zeros((2, 3), np.int64), bq=0)
    assert G.estimate(Q[:0], np.zeros((0, 3), np.int64)).shape == (0, 3, 3)


def test_metric_persists_and_predictor_is_refused(R, pair, tiny_workload, tmp_path):
    m, G, _ = pair
    _, Q = tiny_workload
    p = str(tmp_path / "m.idx")
    G.save(p)
    L = R.Index.load(p)
    assert L.metric == m
    _same(L.search(Q, 10, 4), G.search(Q, 10, 4))
    with pytest.raises(R.RabitqError) as e:
        R.Predictor.train(G, Q, k=10, epochs=1)
    assert e.value.code == R.EUNSUPPORTED
    with pytest.raises(ValueError):
        R.Index.build(Q, 4, seed=1, metric="hamming")
