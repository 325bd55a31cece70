"""Parity of the CUDA path (through the C-ABI) with the CPU oracle.

Bit-exact: the rotation P, k-means centroids and assignment, bucket layout,
codes and factors, probe lists, rotated queries, quantized bit-planes and
their constants, integer inner products, estimated distances and bounds, the
threshold tau, the survivor sets, and the final top-k ids and distances.
The numerics contract that makes bit-exactness possible (canonical FP32
summation order, no contraction, Philox draws) is followed independently by
both sides.
"""
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


@pytest.fixture(scope="module")
def tiny_gpu_index(R, tiny_workload):
    data, _ = tiny_workload
    return R.Index.build(data, 16, seed=2, kmeans_iters=10)


def _u64(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("dpad", [64, 128, 256, 1024])
def test_rotation_bit_exact(R, oracle_mod, dpad):
    P = R.sample_rotation(2, dpad)
    Po = oracle_mod.sample_rotation(2, dpad)
    assert np.array_equal(P.view(np.uint64), Po.view(np.uint64))
    assert np.abs(P @ P.T - np.eye(dpad)).max() <= 1e-13


def test_build_bit_exact(R, oracle_mod, tiny_gpu_index, tiny_oracle_index):
    G, O = tiny_gpu_index, tiny_oracle_index
    assert (G.n, G.d, G.dpad, G.K) == (O.n, O.d, O.dpad, O.K)
    assert np.array_equal(G.centroids().view(np.uint32), O.centroids.view(np.uint32))
    assert np.array_equal(G.assign(), O.assign)
    assert np.array_equal(G.rotation().view(np.uint64), O.P.view(np.uint64))
    assert np.array_equal(G.codes(), O.codes)
    assert np.array_equal(G.factors().view(np.uint32), O.factors.view(np.uint32))
    off, ids = G.buckets()
    assert np.array_equal(off, O.bucket_off)
    assert np.array_equal(ids, O.bucket_ids)


def _compare_trace(G, O, t, i, q, qid, k, nprobe, bq=4, eps0=1.9, seed=3):
    o = O.trace(q, qid, k, nprobe, bq=bq, eps0=eps0, seed=seed)
    npb = min(nprobe, O.K)
    assert np.array_equal(t["probe_ids"][i].cpu().numpy(), o["probe_ids"])
    assert np.array_equal(t["probe_dist"][i].cpu().numpy().view(np.uint32),
                          o["probe_dist"].view(np.uint32))
    assert np.array_equal(t["rq"][i].cpu().numpy().view(np.uint32), o["rq"].view(np.uint32))
    assert np.array_equal(_u64(t["planes"][i]), o["planes"])
    assert np.array_equal(t["sum_qu"][i].cpu().numpy(), o["sum_qu"])
    assert np.array_equal(t["meta"][i].cpu().numpy().view(np.uint32),
                          o["meta"][:, :4].view(np.uint32))
    n = int(t["n_pairs"][i])
    assert n == len(o["pair_id"])
    assert np.array_equal(t["pair_id"][i, :n].cpu().numpy(), o["pair_id"])
    assert np.array_equal(t["pair_ip"][i, :n].cpu().numpy(), o["pair_ip"])
    assert np.array_equal(t["pair_est"][i, :n].cpu().numpy().view(np.uint32),
                          o["pair_est"].view(np.uint32))
    for key in ("tau", "tau_ub", "tau1"):
        assert np.float32(t[key][i].item()).view(np.uint32) == np.float32(o[key]).view(np.uint32), key
    ns = int(t["n_surv"][i])
    assert ns == len(o["surv_ids"])
    assert np.array_equal(np.sort(t["surv_ids"][i, :ns].cpu().numpy()), o["surv_ids"])
    assert np.array_equal(t["ids"][i].cpu().numpy(), o["ids"])
    assert np.array_equal(t["dist"][i].cpu().numpy().view(np.uint32), o["dist"].view(np.uint32))


@pytest.mark.parametrize("k,nprobe,bq,eps0", [(10, 4, 4, 1.9), (10, 16, 4, 1.9), (1, 1, 1, 0.0),
                                               (25, 3, 8, 3.0)])
def test_search_trace_bit_exact(R, tiny_gpu_index, tiny_oracle_index, tiny_workload, k, nprobe,
                                bq, eps0):
    import torch
    _, Q = tiny_workload
    sel = np.array([0, 3, 17, 42, 99])
    qd = torch.from_numpy(Q).cuda()
    t = R.Index.search_trace(tiny_gpu_index, qd, k, nprobe, bq=bq, eps0=eps0,
                             pair_cap=12000, surv_cap=12000)
    for i in sel:
        _compare_trace(tiny_gpu_index, tiny_oracle_index, t, i, Q[i], int(i), k, nprobe, bq, eps0)


def test_search_end_to_end_identical(R, tiny_gpu_index, tiny_oracle_index, tiny_workload):
    import torch
    _, Q = tiny_workload
    ids_o, dist_o = tiny_oracle_index.search(Q, 10, 4)
    ids_h, dist_h = tiny_gpu_index.search(Q, 10, 4)                  # host buffers
    ids_d, dist_d = tiny_gpu_index.search(torch.from_numpy(Q).cuda(), 10, 4)  # device
    assert np.array_equal(ids_h, ids_o)
    assert np.array_equal(dist_h.view(np.uint32), dist_o.view(np.uint32))
    assert np.array_equal(ids_d.cpu().numpy(), ids_o)
    assert np.array_equal(dist_d.cpu().numpy().view(np.uint32), dist_o.view(np.uint32))
    ids2, dist2 = tiny_gpu_index.search(Q, 10, 4)                    # deterministic
    assert np.array_equal(ids2, ids_h) and np.array_equal(dist2, dist_h)


def test_all_buckets_and_padding(R, tiny_gpu_index, tiny_oracle_index, tiny_workload):
    _, Q = tiny_workload
    for k, nprobe in ((10, 16), (1000, 1)):
        ids_o, dist_o = tiny_oracle_index.search(Q[:20], k, nprobe)
        ids_g, dist_g = tiny_gpu_index.search(Q[:20], k, nprobe)
        assert np.array_equal(ids_g, ids_o)
        assert np.array_equal(dist_g.view(np.uint32), dist_o.view(np.uint32))
    assert (ids_g == -1).any() and np.isinf(dist_g[ids_g == -1]).all()


def test_largest_k_matches_oracle(R, tiny_gpu_index, tiny_oracle_index, tiny_workload):
    """k = 1024, the largest the API takes (and 1023): a 4096-code pilot,
    a top-k buffer cut back to k several times during the re-rank, and
    1024-key sorts, in every form of the CTA kernel, the bucket-major
    tensor-core scan, split mode and a search plan."""
    import torch
    _, Q = tiny_workload
    Q = Q[:40]
    qd = torch.from_numpy(Q).cuda()
    G = tiny_gpu_index
    for k, nprobe in ((1024, 16), (1024, 6), (1023, 3)):
        ids_o, dist_o = tiny_oracle_index.search(Q, k, nprobe)
        assert (ids_o >= 0).all()
        for kw in (dict(layout=R.LAYOUT_CTA, staging=R.STAGING_OFF),
                   dict(layout=R.LAYOUT_CTA, staging=R.STAGING_BULK), dict(scan_path=R.SCAN_TC)):
            ids, dist = G.search(qd, k, nprobe, **kw)
            assert np.array_equal(ids.cpu().numpy(), ids_o), (k, nprobe, kw)
            assert np.array_equal(dist.cpu().numpy().view(np.uint32), dist_o.view(np.uint32))
        for nq in (1, 3):                      # small batches: split mode
            ids, dist = G.search(Q[:nq], k, nprobe)
            assert np.array_equal(ids, ids_o[:nq])
            assert np.array_equal(dist.view(np.uint32), dist_o[:nq].view(np.uint32))
    plan = R.Plan(G, 1024, 16, len(Q))
    plan.queries.copy_(qd)
    plan.run(len(Q))
    plan.sync()
    ids_o, dist_o = tiny_oracle_index.search(Q, 1024, 16)
    assert np.array_equal(plan.ids.cpu().numpy(), ids_o)
    assert np.array_equal(plan.dist.cpu().numpy().view(np.uint32), dist_o.view(np.uint32))


def _ragged_case(oracle_mod, n, d, K, code_bits, seed, sample=0):
    rng = np.random.default_rng(seed)
    data = (rng.standard_normal((n, d)) * rng.uniform(0.1, 3, d)).astype(np.float32)
    data[5] = data[6]           # duplicate points (distance ties)
    Q = (rng.standard_normal((7, d)) * 2).astype(np.float32)
    Q[3] = data[11]             # a query equal to a data point
    return data, Q


@pytest.mark.parametrize("n,d,K,code_bits,sample", [(1037, 100, 7, 0, 0), (777, 960, 5, 1024, 0),
                                                    (3001, 33, 40, 128, 1500), (300, 8, 300, 0, 0)])
def test_ragged_shapes_bit_exact(R, oracle_mod, n, d, K, code_bits, sample):
    data, Q = _ragged_case(oracle_mod, n, d, K, code_bits, n + d)
    G = R.Index.build(data, K, seed=5, code_bits=code_bits, kmeans_iters=4, kmeans_sample=sample)
    O = oracle_mod.OracleIndex(data, K=K, seed=5, dpad=G.dpad, iters=4, sample=sample)
    assert np.array_equal(G.centroids().view(np.uint32), O.centroids.view(np.uint32))
    assert np.array_equal(G.assign(), O.assign)
    assert np.array_equal(G.codes(), O.codes)
    assert np.array_equal(G.factors().view(np.uint32), O.factors.view(np.uint32))
    nprobe = min(3, K)
    ids_o, dist_o = O.search(Q, 5, nprobe)
    ids_g, dist_g = G.search(Q, 5, nprobe)
    assert np.array_equal(ids_g, ids_o)
    assert np.array_equal(dist_g.view(np.uint32), dist_o.view(np.uint32))


def test_given_centroids_and_zero_residuals(R, oracle_mod, tiny_workload):
    """Every point its own centroid: zero residuals, a_o := 1, exact estimates."""
    data = tiny_workload[0][:200]
    G = R.Index.build(data, 200, seed=3, centroids=data)
    O = oracle_mod.OracleIndex(data, K=200, seed=3, centroids=data)
    assert np.array_equal(G.assign(), O.assign)
    assert np.array_equal(G.factors().view(np.uint32), O.factors.view(np.uint32))
    assert (G.factors()[:, 0] == 0).all()
    ids_g, dist_g = G.search(data[:10], 3, 5)
    ids_o, dist_o = O.search(data[:10], 3, 5)
    assert np.array_equal(ids_g, ids_o) and (ids_g[:, 0] == np.arange(10)).all()


def test_save_load_roundtrip(R, tiny_gpu_index, tiny_workload, tmp_path):
    _, Q = tiny_workload
    p = str(tmp_path / "tiny.idx")
    tiny_gpu_index.save(p)
    L = R.Index.load(p)
    assert np.array_equal(L.codes(), tiny_gpu_index.codes())
    a = tiny_gpu_index.search(Q, 10, 4)
    b = L.search(Q, 10, 4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    raw = bytearray(open(p, "rb").read())
    raw[-5] ^= 0xFF
    open(p, "wb").write(bytes(raw))
    with pytest.raises(R.RabitqError) as e:
        R.Index.load(p)
    assert e.value.code == R.EIO


def test_invalid_search_arguments(R, tiny_gpu_index, tiny_workload):
    _, Q = tiny_workload
    for kw in (dict(k=0, nprobe=4), dict(k=1025, nprobe=4), dict(k=10, nprobe=17),
               dict(k=10, nprobe=4, bq=9),
               dict(k=10, nprobe=4, eps0=float("nan"))):
        with pytest.raises(R.RabitqError) as e:
            tiny_gpu_index.search(Q, **kw)
        assert e.value.code == R.EINVAL
    ids, dist = tiny_gpu_index.search(Q[:0], 10, 4)
    assert ids.shape == (0, 10)
    bad = Q[:5].copy()
    bad[2, 7] = np.nan
    with pytest.raises(R.RabitqError) as e:
        tiny_gpu_index.search(bad, 10, 4)
    assert e.value.code == R.EINVAL and "non-finite" in str(e.value)
    ids, _ = tiny_gpu_index.search(Q[:5], 10, 4)   # the index is still usable
    assert (ids >= 0).all()


# ------------------------------------------------- tensor-core rotation modes
@pytest.mark.parametrize("n,d,code_bits,nq", [(3000, 128, 0, 100), (2000, 960, 1024, 300),
                                              (1500, 200, 256, 129)])
def test_tensor_core_rotation_error(R, n, d, code_bits, nq):
    """BF16 / TF32 query rotation on tensor cores (FP32 accumulation) against
    the FP64 rotation P^{-1}[q; 0]: normwise relative error per query below
    a few operand ulps (2^-8 BF16, 2^-11 TF32)."""
    import torch
    rng = np.random.default_rng(d)
    data = rng.standard_normal((n, d)).astype(np.float32)
    Q = (rng.standard_normal((nq, d)) * 3).astype(np.float32)
    G = R.Index.build(data, 8, seed=4, code_bits=code_bits, kmeans_iters=2)
    P = G.rotation()
    ref = Q.astype(np.float64) @ P[:d]
    qd = torch.from_numpy(Q).cuda()
    fp32 = G.search_trace(qd, 5, 2)["rq"].cpu().numpy().astype(np.float64)
    assert np.abs(fp32 - ref).max() <= 1e-5 * np.abs(ref).max()
    for mode, tol in ((R.ROT_BF16, 8e-3), (R.ROT_TF32, 1.2e-3)):
        rq = G.search_trace(qd, 5, 2, rot_precision=mode)["rq"].cpu().numpy().astype(np.float64)
        err = np.linalg.norm(rq - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() <= tol, (mode, err.max())
        assert err.mean() >= 1e-7  # the reduced precision is really in effect


def test_tensor_core_rotation_search(R, tiny_gpu_index, tiny_workload):
    _, Q = tiny_workload
    ids32, _ = tiny_gpu_index.search(Q, 10, 4)
    for mode in (R.ROT_BF16, R.ROT_TF32):
        ids, dist = tiny_gpu_index.search(Q, 10, 4, rot_precision=mode)
        agree = np.mean([len(set(a) & set(b)) / 10 for a, b in zip(ids.tolist(), ids32.tolist())])
        assert agree >= 0.98, (mode, agree)
        assert (np.diff(dist, axis=1) >= 0).all()


# --------------------------------------------- tensor-core (bucket-major) scan
def _paths_identical(R, G, Q, k, nprobe, **kw):
    a = G.search(Q, k, nprobe, scan_path=R.SCAN_POPC, **kw)
    b = G.search(Q, k, nprobe, scan_path=R.SCAN_TC, **kw)
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))
    return b


@pytest.mark.parametrize("k,nprobe", [(10, 4), (1, 1), (100, 16), (25, 3)])
def test_tc_scan_matches_popcount_and_oracle(R, tiny_gpu_index, tiny_oracle_index, tiny_workload,
                                              k, nprobe):
    """The tensor-core scan (codes x queries per bucket, BF16 0/1 x 0..15,
    FP32 accumulation) returns exactly what the popcount scan and the oracle
    return: integer inner products are exact, the rest is the same arithmetic."""
    _, Q = tiny_workload
    ids, dist = _paths_identical(R, tiny_gpu_index, Q, k, nprobe)
    ids_o, dist_o = tiny_oracle_index.search(Q, k, nprobe)
    assert np.array_equal(ids, ids_o)
    assert np.array_equal(dist.view(np.uint32), dist_o.view(np.uint32))


def test_tc_scan_trace_matches(R, tiny_gpu_index, tiny_workload):
    import torch
    _, Q = tiny_workload
    qd = torch.from_numpy(Q).cuda()
    G = tiny_gpu_index
    a = G.search_trace(qd, 10, 6, surv_cap=12000)
    b = G.search_trace(qd, 10, 6, surv_cap=12000, scan_path=R.SCAN_TC)
    for key in ("tau_ub", "tau1", "tau", "n_surv", "n_pairs", "ids", "dist", "probe_ids"):
        assert torch.equal(a[key], b[key]), key
    for i in range(len(Q)):
        n = int(a["n_surv"][i])
        assert torch.equal(torch.sort(a["surv_ids"][i, :n]).values,
                           torch.sort(b["surv_ids"][i, :n]).values)


@pytest.mark.parametrize("n,d,code_bits,K,nq,k,nprobe", [
    (20000, 128, 0, 16, 2000, 10, 4),      # 5 M tiles x 4 N tiles per bucket
    (6000, 960, 1024, 8, 300, 20, 3),      # D' = 1024: 16 K stages
    (5000, 200, 256, 64, 700, 50, 12),     # D' = 256, ragged buckets
])
def test_tc_scan_shapes(R, oracle_mod, n, d, code_bits, K, nq, k, nprobe):
    rng = np.random.default_rng(n + d)
    cen = rng.standard_normal((30, d))
    data = (cen[rng.integers(0, 30, n)] + 0.4 * rng.standard_normal((n, d))).astype(np.float32)
    Q = (cen[rng.integers(0, 30, nq)] + 0.4 * rng.standard_normal((nq, d))).astype(np.float32)
    G = R.Index.build(data, K, seed=6, code_bits=code_bits, kmeans_iters=3)
    ids, dist = _paths_identical(R, G, Q, k, nprobe)
    O = oracle_mod.OracleIndex(data, K=K, seed=6, dpad=G.dpad, iters=3, threads=8)
    ids_o, dist_o = O.search(Q, k, nprobe, threads=8)   # query indices key the rounding
    assert np.array_equal(ids, ids_o)
    assert np.array_equal(dist.view(np.uint32), dist_o.view(np.uint32))
