"""Pins of the oracle's inner-product / cosine metric and of its
single-code estimator against the mathematics.

The inner-product form follows the closing footnote of the paper (§6):
<o, q> = ||o - c|| ||q - c|| <o', q'> + <o, c> + <q, c> - ||c||^2 with unit
o' = (o - c)/||o - c||, q' likewise, so the same code and the same estimator
of <o', q'> (Theorem 3.2) serve both metrics. Each check compares the oracle
with something other than itself: FP64 numpy definitions, the already pinned
squared-distance path, or brute force.
"""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def pair_indices(oracle_mod, tiny_workload, tiny_oracle_index):
    """An inner-product index on the same data, centroids and P as the
    squared-distance index (so both hold the same codes)."""
    data, _ = tiny_workload
    L2 = tiny_oracle_index
    IP = oracle_mod.OracleIndex(data, K=L2.K, seed=2, centroids=L2.centroids, P=L2.P,
                                metric="ip")
    return L2, IP


def _recall(a, b):
    return np.mean([len(set(x) & set(y)) / len(y) for x, y in zip(a.tolist(), b.tolist())])


def test_normalize_rows(oracle_mod):
    rng = np.random.default_rng(1)
    x = (rng.standard_normal((50, 37)) * rng.uniform(0.01, 100, (50, 1))).astype(np.float32)
    x[7] = 0
    u = oracle_mod.normalize_rows(x)
    n64 = np.linalg.norm(u.astype(np.float64), axis=1)
    assert np.all(np.abs(n64[np.arange(50) != 7] - 1) <= 1e-6)
    assert np.all(u[7] == 0)
    cos = (u.astype(np.float64) * x).sum(1) / np.maximum(np.linalg.norm(x.astype(np.float64), axis=1), 1e-30)
    assert np.all(np.abs(cos[np.arange(50) != 7] - 1) <= 1e-6)


def test_ip_factors_definition(pair_indices):
    """Same codes; F2 and F3 exactly half of the distance form's (the score's
    coefficient and bound are half those of the squared distance);
    F1 = -<o_r - c, c> in FP64."""
    L2, IP = pair_indices
    assert np.array_equal(L2.codes, IP.codes)
    assert np.array_equal(L2.factors[:, 3], IP.factors[:, 3])
    assert np.array_equal(IP.factors[:, 1], L2.factors[:, 1] * np.float32(0.5))
    assert np.array_equal(IP.factors[:, 2], L2.factors[:, 2] * np.float32(0.5))
    c = L2.centroids[L2.assign].astype(np.float64)
    res = L2.data.astype(np.float64) - c
    want = -(res * c).sum(1)
    scale = np.abs(res).sum(1) * np.abs(c).max(1) + 1e-30
    assert np.all(np.abs(IP.factors[:, 0] - want) <= 1e-5 * scale)


def test_ip_estimate_is_the_distance_identity(pair_indices, tiny_workload):
    """<o, q> = (||o||^2 + ||q||^2 - ||o - q||^2) / 2 holds for the estimates
    too (same code, same quantized query): the inner-product estimate equals
    (||o||^2 + ||q||^2 - distance estimate) / 2 and its bound is half the
    distance bound, up to FP32 rounding."""
    L2, IP = pair_indices
    _, Q = tiny_workload
    rng = np.random.default_rng(4)
    ids = rng.integers(0, L2.n, (30, 64))
    el2 = L2.estimate(Q[:30], ids).astype(np.float64)
    eip = IP.estimate(Q[:30], ids).astype(np.float64)
    o2 = (L2.data.astype(np.float64) ** 2).sum(1)[ids]
    q2 = (Q[:30].astype(np.float64) ** 2).sum(1)[:, None]
    want = (o2 + q2 - el2[..., 0]) / 2
    scale = o2 + q2 + np.abs(el2[..., 0])
    assert np.all(np.abs(eip[..., 0] - want) <= 4e-6 * scale)
    b_l2 = el2[..., 2] - el2[..., 0]
    b_ip = eip[..., 2] - eip[..., 0]
    assert np.all(np.abs(b_ip - b_l2 / 2) <= 4e-6 * scale)
    assert np.all(np.abs((eip[..., 0] - eip[..., 1]) - b_l2 / 2) <= 4e-6 * scale)


@pytest.mark.parametrize("metric", ["l2", "ip"])
def test_single_code_estimates_equal_the_scan(pair_indices, tiny_workload, metric):
    """The single-code estimator quantizes the query against each code's own
    cluster with the same random stream as the bucket scan, so its values are
    bit-identical to the scan's per-pair estimates (trace of the search)."""
    X = pair_indices[0] if metric == "l2" else pair_indices[1]
    _, Q = tiny_workload
    qi = 5
    t = X.trace(Q[qi], qi, 10, 6)
    ids = -np.ones((qi + 1, len(t["pair_id"])), np.int64)
    ids[qi] = t["pair_id"]
    est = X.estimate(Q[:qi + 1], ids)
    assert np.isnan(est[:qi]).all()
    pe = t["pair_est"]
    want = pe if metric == "l2" else -pe[:, [0, 2, 1]]
    assert np.array_equal(est[qi].view(np.uint32), want.astype(np.float32).view(np.uint32))


def test_ip_estimator_unbiased_and_bounded(pair_indices, tiny_workload):
    """Estimated inner products against FP64 truth: unbiased (least-squares
    slope 1, intercept 0) and inside the bound for most pairs at eps0 = 1.9
    (Theorem 3.2)."""
    _, IP = pair_indices
    _, Q = tiny_workload
    rng = np.random.default_rng(6)
    ids = rng.integers(0, IP.n, (60, 200))
    est = IP.estimate(Q[:60], ids).astype(np.float64)
    true = np.einsum("ijd,id->ij", IP.data[ids].astype(np.float64), Q[:60].astype(np.float64))
    span = true.max() - true.min()
    slope, icpt = np.polyfit(((true - true.mean()) / span).ravel(),
                             ((est[..., 0] - true.mean()) / span).ravel(), 1)
    assert abs(slope - 1) <= 0.02 and abs(icpt) <= 0.01
    inside = (est[..., 1] <= true) & (true <= est[..., 2])
    assert inside.mean() >= 0.85
    # the centroid terms are exact, so the error is that of the <o', q'>
    # estimate scaled by ||o - c|| ||q - c||: O(1/sqrt(D')) (Theorem 3.2)
    c = IP.centroids[IP.assign[ids]].astype(np.float64)
    n_o = np.linalg.norm(IP.data[ids].astype(np.float64) - c, axis=2)
    n_q = np.linalg.norm(Q[:60, None, :].astype(np.float64) - c, axis=2)
    rel = np.abs(est[..., 0] - true) / (n_o * n_q)
    assert np.median(rel) <= 1 / np.sqrt(IP.dpad - 1)


def test_ip_probes_largest_inner_products(pair_indices, tiny_workload):
    _, IP = pair_indices
    _, Q = tiny_workload
    for qi in (0, 9):
        t = IP.trace(Q[qi], qi, 10, 5)
        s = -(IP.centroids.astype(np.float64) @ Q[qi].astype(np.float64))
        want = np.lexsort((np.arange(IP.K), s))[:5]
        assert np.array_equal(t["probe_ids"], want)


def test_ip_search_is_exact_mips_without_pruning(oracle_mod, pair_indices, tiny_workload):
    """With every bucket probed and a bound too wide to drop anything, the
    search returns the exact maximum-inner-product top-k (FP64 numpy)."""
    _, IP = pair_indices
    _, Q = tiny_workload
    ids, ip = IP.search(Q[:40], 10, IP.K, eps0=1e4)
    true = Q[:40].astype(np.float64) @ IP.data.astype(np.float64).T
    want = np.argsort(-true, axis=1, kind="stable")[:, :10]
    got_vals = np.take_along_axis(true, ids, 1)
    want_vals = np.take_along_axis(true, want, 1)
    assert np.all(np.abs(got_vals - want_vals) <= 1e-5 * np.abs(want_vals).max())
    assert np.all(np.abs(ip - got_vals) <= 1e-5 * np.abs(want_vals).max())
    assert np.all(np.diff(ip, axis=1) <= 0)  # descending
    bids, bip = oracle_mod.bruteforce_ip(IP.data, Q[:40], 10)
    assert np.array_equal(ids, bids) and np.array_equal(ip, bip)


def test_ip_search_recall_at_eps0(oracle_mod, pair_indices, tiny_workload):
    """Near-exact recall at eps0 = 1.9 with every bucket probed (§5.2.4);
    dropping the bound (eps0 = 0) loses recall."""
    _, IP = pair_indices
    _, Q = tiny_workload
    gt, _ = oracle_mod.bruteforce_ip(IP.data, Q, 10)
    ids, _ = IP.search(Q, 10, IP.K)
    r = _recall(ids, gt)
    assert r >= 0.99
    ids0, _ = IP.search(Q, 10, IP.K, eps0=0.0)
    assert _recall(ids0, gt) < r
    ids1, _ = IP.search(Q, 10, IP.K, mode=1)
    assert _recall(ids1, gt) >= 0.99


def test_cosine_search(oracle_mod, tiny_workload):
    """Cosine = inner product of unit vectors: results are the exact top-k
    cosine similarities (FP64 numpy) when nothing is pruned."""
    data, Q = tiny_workload
    X = oracle_mod.OracleIndex(data, K=16, seed=2, iters=5, metric="cosine")
    ids, cs = X.search(Q[:30], 10, X.K, eps0=1e4)
    d64 = data.astype(np.float64)
    q64 = Q[:30].astype(np.float64)
    cos = (q64 @ d64.T) / np.linalg.norm(q64, axis=1)[:, None] / np.linalg.norm(d64, axis=1)[None]
    want = np.sort(cos, axis=1)[:, ::-1][:, :10]
    assert np.all(np.abs(np.take_along_axis(cos, ids, 1) - want) <= 2e-6)
    assert np.all(np.abs(cs - want) <= 2e-6)
    idg, _ = X.search(Q, 10, 4)
    gt = np.argsort(-((Q.astype(np.float64) @ d64.T) / np.linalg.norm(d64, axis=1)), 1)[:, :10]
    assert _recall(idg, gt) >= 0.8


@pytest.mark.parametrize("metric", ["ip", "cosine"])
def test_ip_ties_resolve_by_id(oracle_mod, metric):
    """300 identical points along the query hold its 300 largest inner
    products (and cosines), by FP64 brute force: ranked by (-value, id),
    the top-k are the k lowest of their ids, all with one value."""
    rng = np.random.default_rng(31)
    data = rng.standard_normal((3000, 64)).astype(np.float32)
    q = rng.standard_normal(64).astype(np.float32)
    data[500:800] = q * np.float32(3.0)
    Q = np.stack([q, q * np.float32(0.5)])
    d64 = data.astype(np.float64)
    if metric == "cosine":
        d64 = d64 / np.linalg.norm(d64, axis=1, keepdims=True)
    top = np.argsort(-(Q.astype(np.float64) @ d64.T), axis=1, kind="stable")[:, :300]
    assert (np.sort(top, axis=1) == np.arange(500, 800)).all()
    X = oracle_mod.OracleIndex(data, K=12, seed=4, metric=metric)
    for k in (1, 100, 300):
        ids, v = X.search(Q, k, X.K)
        assert (ids == np.arange(500, 500 + k)).all(), (metric, k)
        assert (v == v[:, :1]).all()
