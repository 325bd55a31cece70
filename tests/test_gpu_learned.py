"""Learned probe count on the GPU, through the C-ABI, against the oracle of
oracle/mlp_oracle.py:

* one forward/backward pass: the gradient of every parameter block within a
  normwise FP32 tolerance of the FP64 chain rule; one Adam step likewise,
  with the BF16 working copy the exact rounding of the FP32 master;
* labels (bucket ranks and probe counts): bit-exact;
* features: bit-exact (correctly rounded FP32 ratios of bit-exact canonical
  distances); network outputs within tolerance of FP64; probe counts equal
  to the FP32 decision rule applied to the GPU's outputs;
* the fused inference kernel equals the training forward bit for bit;
* the learned search equals the plain search with the same per-query counts;
* trained on SIFT-shaped data, the predictor reaches recall 0.95 with fewer
  probes on average than the smallest fixed nprobe that does.
"""
import math

import numpy as np
import pytest

from oracle import mlp_oracle as M

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


def bf16_round(x):
    """Round-to-nearest-even to BF16, returned as float32 (bit manipulation)."""
    u = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def rand_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    W1 = rng.uniform(-1, 1, (64, 256)) * math.sqrt(6 / 64) * scale
    W2 = rng.uniform(-1, 1, (256, 256)) * math.sqrt(6 / 256) * scale
    w3 = rng.uniform(-1, 1, 256) * math.sqrt(6 / 256) * scale
    p = M.pack(W1, rng.normal(0, 0.1, 256), W2, rng.normal(0, 0.1, 256), w3, 2.0)
    return bf16_round(p.astype(np.float32))


BLOCKS = [("W1", M.OFF_W1, M.OFF_B1), ("b1", M.OFF_B1, M.OFF_W2), ("W2", M.OFF_W2, M.OFF_B2),
          ("b2", M.OFF_B2, M.OFF_W3), ("w3", M.OFF_W3, M.OFF_B3), ("b3", M.OFF_B3, M.N_PARAMS)]


@pytest.mark.parametrize("B", [1, 37, 300, 1024])
def test_mlp_gradient_matches_oracle(R, B):
    p = rand_params(10 + B)
    rng = np.random.default_rng(B)
    X = rng.uniform(0, 1, (B, 64)).astype(np.float32)
    t = rng.uniform(0, 9, B).astype(np.float32)
    y, g, loss = R.mlp_grad(p, X, t)
    y64, _ = M.forward(p, X)
    g64 = M.backward(p, X, t)
    # FP32 sums of at most 1024 terms: relative error well below 1e-4
    assert np.max(np.abs(y - y64)) <= 1e-4 * (1 + np.max(np.abs(y64)))
    assert loss == pytest.approx(M.loss(p, X, t), rel=1e-4)
    for name, a, b in BLOCKS:
        ref = g64[a:b]
        err = np.linalg.norm(g[a:b] - ref)
        assert err <= 1e-4 * np.linalg.norm(ref) + 1e-7, (name, err, np.linalg.norm(ref))


def test_mlp_gradient_deterministic(R):
    p = rand_params(3)
    X = np.random.default_rng(4).uniform(0, 1, (513, 64)).astype(np.float32)
    t = np.linspace(0, 8, 513).astype(np.float32)
    a = R.mlp_grad(p, X, t)
    b = R.mlp_grad(p, X, t)
    assert np.array_equal(a[0].view(np.uint32), b[0].view(np.uint32))
    assert np.array_equal(a[1].view(np.uint32), b[1].view(np.uint32))


@pytest.mark.parametrize("step", [1, 2, 50])
def test_adam_step_matches_oracle(R, step):
    rng = np.random.default_rng(step)
    n = M.N_PARAMS
    master = rng.normal(0, 0.1, n).astype(np.float32)
    m1 = (rng.normal(0, 1e-3, n) if step > 1 else np.zeros(n)).astype(np.float32)
    m2 = (rng.uniform(0, 1e-6, n) if step > 1 else np.zeros(n)).astype(np.float32)
    g = rng.normal(0, 1e-3, n).astype(np.float32)
    ms, a, b, w = R.mlp_adam(master, m1, m2, g, step, 1e-3)
    # the library's hyper-parameters are the FP32 values of 0.9, 0.999, 1e-3
    f = lambda v: float(np.float32(v))  # noqa: E731
    ms64, a64, b64 = M.adam(master, m1, m2, g, step, f(1e-3), b1=f(0.9), b2=f(0.999), eps=f(1e-8))
    # FP32 rounding of each operation, bounded by the magnitudes of the terms
    # (m1 and the update can cancel, so a relative bound would not hold)
    u = 2.0 ** -24
    m1t = 0.9 * np.abs(m1.astype(np.float64)) + 0.1 * np.abs(g.astype(np.float64))
    assert np.all(np.abs(a - a64) <= 4 * u * m1t + 1e-30)
    assert np.all(np.abs(b - b64) <= 6 * u * b64 + 1e-30)
    # the step lr m1_hat / (sqrt(v_hat) + eps) inherits m1's absolute error
    c1, c2 = 1 - f(0.9) ** step, 1 - f(0.999) ** step
    den = np.sqrt(b64 / c2) + f(1e-8)
    step_err = f(1e-3) * (8 * u * m1t / c1) / den + 8 * u * np.abs(master - ms64)
    assert np.all(np.abs(ms - ms64) <= 2 * u * np.abs(master) + step_err + 1e-30)
    assert np.array_equal(w.view(np.uint32), bf16_round(ms).view(np.uint32))


@pytest.mark.parametrize("k,target,nmax", [(10, 0.9, 16), (10, 1.0, 5), (7, 0.5, 16), (1, 1.0, 3)])
def test_labels_bit_exact(R, oracle_mod, tiny_workload, tiny_gpu_index, tiny_oracle_index,
                          k, target, nmax):
    data, queries = tiny_workload
    gt, _ = oracle_mod.bruteforce_knn(data, queries, k, threads=8)
    gt = gt.copy()
    gt[::9, -1] = -1  # a few missing neighbours
    ranks, lab = tiny_gpu_index.compute_labels(queries, gt, k, target, nmax)
    O = tiny_oracle_index
    ranks_o, lab_o = M.labels(queries, O.centroids, O.assign, gt, k, target, nmax)
    assert np.array_equal(ranks, ranks_o)
    assert np.array_equal(lab, lab_o)


def _predictor_from_params(R, p, s0, mult, nmax, K):
    return R.Predictor.create(p, s0, mult, nmax, K)


@pytest.mark.parametrize("K,nq", [(16, 100), (300, 77)])
def test_predict_matches_oracle(R, oracle_mod, tiny_workload, K, nq):
    data, queries = tiny_workload
    queries = queries[:nq] if nq <= len(queries) else queries
    idx = R.Index.build(data, K, seed=2, kmeans_iters=3) if K != 16 else None
    if idx is None:
        idx = R.Index.build(data, 16, seed=2, kmeans_iters=10)
    C = idx.centroids()
    p = rand_params(21, scale=0.5)
    s0, mult, nmax = 40.0, 1.3, min(K, 200)
    pr = _predictor_from_params(R, p, s0, mult, nmax, K)
    npb, feat, y = idx.predict_nprobe(pr, queries, features=True)
    # features: bit-exact from the oracle's canonical distances and selection
    _, dsel = M.nearest_buckets(queries, C, 64)
    Xo = M.features(dsel, s0)
    assert np.array_equal(feat.view(np.uint32), Xo.view(np.uint32))
    # network output: FP32 vs FP64
    y64, _ = M.forward(p, Xo)
    assert np.max(np.abs(y - y64)) <= 1e-4 * (1 + np.max(np.abs(y64)))
    # the probe-count decision in FP32 on the GPU's outputs
    assert np.array_equal(npb, M.probe_count(y, mult, nmax))
    # and on the FP64 outputs, except within rounding of a boundary
    np64 = M.probe_count(y64, mult, nmax)
    v = mult * np.exp2(np.minimum(y64, 30))
    near = np.abs(v - np.rint(v)) < 1e-4 * v
    assert np.array_equal(npb[~near], np64[~near])


def test_inference_equals_training_forward(R, tiny_workload, tiny_gpu_index):
    _, queries = tiny_workload
    p = rand_params(5)
    pr = R.Predictor.create(p, 10.0, 1.0, 16, 16)
    npb, feat, y = tiny_gpu_index.predict_nprobe(pr, queries, features=True)
    y2, _, _ = R.mlp_grad(p, feat, np.zeros(len(queries), np.float32))
    assert np.array_equal(y.view(np.uint32), y2.view(np.uint32))


@pytest.mark.parametrize("scan", ["popc", "tc"])
@pytest.mark.parametrize("nmax", [12, 16])  # 16 = K: features read from the probe list
def test_search_learned_equals_per_query_search(R, tiny_workload, tiny_gpu_index, scan, nmax):
    import torch
    _, queries = tiny_workload
    p = rand_params(8, scale=1.0)
    pr = R.Predictor.create(p, 30.0, 1.0, nmax, 16)
    path = R.SCAN_POPC if scan == "popc" else R.SCAN_TC
    npb = tiny_gpu_index.predict_nprobe(pr, queries)
    assert npb.min() >= 1 and npb.max() <= nmax and len(np.unique(npb)) > 1
    ids, dist = tiny_gpu_index.search_learned(pr, queries, 10, scan_path=path)
    ids2, dist2 = tiny_gpu_index.search(queries, 10, nmax, per_query_nprobe=npb, scan_path=path)
    assert np.array_equal(ids, ids2)
    assert np.array_equal(dist.view(np.uint32), dist2.view(np.uint32))
    # device queries give the same
    qd = torch.from_numpy(queries).cuda()
    idd, dd = tiny_gpu_index.search_learned(pr, qd, 10, scan_path=path)
    assert np.array_equal(idd.cpu().numpy(), ids)


def test_per_query_nprobe_matches_oracle(R, tiny_workload, tiny_gpu_index, tiny_oracle_index):
    """Each query probes its own count: the oracle's search of query i (its
    own Philox query id i) with nprobe_i gives the same ids and distances."""
    _, queries = tiny_workload
    npb = (np.arange(len(queries)) % 16 + 1).astype(np.int32)
    for path in (R.SCAN_POPC, R.SCAN_TC):
        ids, dist = tiny_gpu_index.search(queries, 10, 16, per_query_nprobe=npb, scan_path=path)
        for i in range(0, len(queries), 3):
            o = tiny_oracle_index.trace(queries[i], i, 10, int(npb[i]))
            assert np.array_equal(ids[i], o["ids"]), (path, i)
            assert np.array_equal(dist[i].view(np.uint32), o["dist"].view(np.uint32)), (path, i)


def test_predictor_api_errors(R, tiny_gpu_index, tiny_workload):
    _, queries = tiny_workload
    p = rand_params(1)
    with pytest.raises(R.RabitqError):
        R.Predictor.create(p, 0.0, 1.0, 8, 16)          # s0 must be > 0
    with pytest.raises(R.RabitqError):
        R.Predictor.create(p, 1.0, 1.0, 17, 16)         # nprobe_max > K
    bad = p.copy()
    bad[5] = np.nan
    with pytest.raises(R.RabitqError):
        R.Predictor.create(bad, 1.0, 1.0, 8, 16)
    pr = R.Predictor.create(p, 1.0, 1.0, 8, 32)          # made for K = 32
    with pytest.raises(R.RabitqError):
        tiny_gpu_index.search_learned(pr, queries, 10)
    with pytest.raises(R.RabitqError):
        R.Predictor.train(tiny_gpu_index, queries[:1], k=10)   # fewer than 2 queries
    with pytest.raises(R.RabitqError):
        R.Predictor.train(tiny_gpu_index, queries, k=10, target_recall=1.5)


def test_train_on_tiny_is_deterministic(R, tiny_gpu_index, tiny_workload):
    from paper_2405_12497_gb300 import synth
    _, train_q = synth.make(synth.TINY, nq=2000, seed_query=7)
    a = R.Predictor.train(tiny_gpu_index, train_q, k=10, nprobe_max=16, epochs=3, batch=256)
    b = R.Predictor.train(tiny_gpu_index, train_q, k=10, nprobe_max=16, epochs=3, batch=256)
    assert np.array_equal(a.params().view(np.uint32), b.params().view(np.uint32))
    ia = a.info()
    assert ia["n_train"] + ia["n_val"] == 2000 and ia["n_val"] == 200
    assert ia["val_recall"] >= 0.95 - 1e-6
    assert 1.0 <= ia["val_mean_nprobe"] <= 16.0
    assert np.all(bf16_round(a.params()) == a.params())


def test_learned_beats_fixed_nprobe(R, oracle_mod):
    """SIFT-shaped 200k x 128, K = 1024, k = 100. Both operating points are
    chosen on 2000 calibration queries (the smallest fixed nprobe and the
    smallest multiplier 2^(i/32) whose calibration recall@100 reaches 0.955),
    then frozen and evaluated once on 2000 other (held-out) queries: both
    reach recall@100 >= 0.95 there, and the learned search probes fewer
    buckets and runs faster (search plans, best of five) than the fixed one
    on a batch of 8000 held-out queries (at a few thousand queries the
    learned plan's own fixed cost, the network and its probe lists, is a
    large share of a sub-millisecond search)."""
    import torch
    from paper_2405_12497_gb300 import synth
    w = synth.SIFT_LIKE
    data, queries = synth.make(w, n=200_000, nq=2000)
    _, cal_q = synth.make(w, n=200_000, nq=2000, seed_query=11, with_data=False)
    _, train_q = synth.make(w, n=200_000, nq=40_000, seed_query=7, with_data=False)
    idx = R.Index.build(data, 1024, seed=2, kmeans_iters=10)
    truth, _ = oracle_mod.bruteforce_knn(data, queries, 100, threads=16)
    cal_truth, _ = oracle_mod.bruteforce_knn(data, cal_q, 100, threads=16)

    def recall(ids, gt):
        return np.mean([len(np.intersect1d(ids[i], gt[i])) / 100 for i in range(len(ids))])

    cal_target = 0.955
    fixed = None
    for npb in range(8, 257, 4):
        ids, _ = idx.search(cal_q, 100, npb)
        if recall(ids, cal_truth) >= cal_target:
            fixed = npb
            break
    assert fixed is not None
    pr = R.Predictor.train(idx, train_q, k=100, target_recall=0.95, nprobe_max=256, epochs=20)
    def cal_rec(i):
        pr.set_mult(2.0 ** (i / 32))
        ids, _ = idx.search_learned(pr, cal_q, 100)
        return recall(ids, cal_truth)

    lo, hi = -128, 255                                    # bisection on the grid
    assert cal_rec(hi) >= cal_target
    while lo < hi:
        mid = (lo + hi) // 2
        if cal_rec(mid) >= cal_target:
            hi = mid
        else:
            lo = mid + 1
    mult = 2.0 ** (lo / 32)
    pr.set_mult(mult)                                    # frozen from here on
    ids_f, _ = idx.search(queries, 100, fixed)
    ids_l, _ = idx.search_learned(pr, queries, 100)
    rec_f, rec_l = recall(ids_f, truth), recall(ids_l, truth)
    mean_np = idx.predict_nprobe(pr, queries).mean()
    _, time_q = synth.make(w, n=200_000, nq=8000, seed_query=13, with_data=False)
    qd = torch.from_numpy(time_q).cuda()

    def best_ms(plan):
        plan.queries.copy_(qd)
        times = []
        for _ in range(6):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan.run(len(time_q))
            e1.record()
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        plan.sync()
        return min(times[1:])

    t_f = best_ms(R.Plan(idx, 100, fixed, len(time_q)))
    t_l = best_ms(R.Plan(idx, 100, 0, len(time_q), predictor=pr))
    print(f"fixed nprobe {fixed}: recall {rec_f:.4f}, {t_f:.3f} ms; learned (mult {mult:.3f}, "
          f"mean nprobe {mean_np:.1f}): recall {rec_l:.4f}, {t_l:.3f} ms")
    assert rec_f >= 0.95 and rec_l >= 0.95
    assert mean_np < fixed
    assert t_l < t_f
