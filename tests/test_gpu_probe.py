"""The IVF probe lists (§4) from tensor-core scores with exact refinement are
bit-identical to a full canonical scan (the oracle's select over canonical
FP32 scores), including inputs built to defeat the filter: wide value
ranges, near-equal centroid distances (the candidate list overflows and the
exact fallback runs) and the inner-product metric.
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


def _probe_lists(R, G, Q, nprobe):
    import torch
    t = R.Index.search_trace(G, torch.from_numpy(Q).cuda(), 1, nprobe)
    return t["probe_ids"].cpu().numpy(), t["probe_dist"].cpu().numpy()


def _check(R, oracle_mod, data, cents, Q, nprobe, metric="l2"):
    G = R.Index.build(data, cents.shape[0], seed=1, centroids=cents, metric=metric)
    O = oracle_mod.OracleIndex(data, K=cents.shape[0], seed=1, centroids=cents, metric=metric)
    ids, dist = _probe_lists(R, G, Q, nprobe)
    for i in range(Q.shape[0]):
        t = O.trace(Q[i], i, 1, nprobe)  # (the oracle makes cosine queries unit itself)
        assert np.array_equal(ids[i], t["probe_ids"]), (i, ids[i][:8], t["probe_ids"][:8])
        assert np.array_equal(dist[i].view(np.uint32), t["probe_dist"].view(np.uint32))


# (33, 300, 1e-3, 100): more probes than the 24 pooled keys, so the threshold
# comes from the histogram of all keys; (8, 16384, 1.0, 1000): most groups of
# 128 centroids hold 8 keys under the threshold, so all keys are scanned
@pytest.mark.parametrize("d,K,scale,nprobe", [(8, 7, 1.0, 7), (33, 300, 1e-3, 17),
                                               (33, 300, 1e-3, 100), (128, 1024, 200.0, 64),
                                               (100, 2000, 1e3, 1), (8, 16384, 1.0, 1000)])
def test_probe_lists_match_full_scan(R, oracle_mod, d, K, scale, nprobe):
    rng = np.random.default_rng(d + K)
    cents = (rng.standard_normal((K, d)) * scale * rng.uniform(0.2, 2, d)).astype(np.float32)
    data = cents + (rng.standard_normal((K, d)) * 0.1 * scale).astype(np.float32)
    Q = (rng.standard_normal((24, d)) * scale).astype(np.float32)
    Q[0] = cents[3]              # a query on a centroid
    Q[1] = 0                     # the zero query
    _check(R, oracle_mod, data, cents, Q, nprobe)


def test_crowded_group_is_scanned_in_full(R, oracle_mod):
    """The 64 nearest centroids of some queries have ids 0..63 (one group of
    128 centroids): that group's 8 pooled keys are all under the threshold,
    so its keys are scanned in full; the other queries take their
    candidates from the pool."""
    rng = np.random.default_rng(11)
    d, K = 16, 1024
    cents = rng.standard_normal((K, d)).astype(np.float32)
    Q = rng.standard_normal((12, d)).astype(np.float32)
    cents[:64] = Q[2] + 0.05 * rng.standard_normal((64, d)).astype(np.float32)
    cents[64:80] = Q[5] + 0.05 * rng.standard_normal((16, d)).astype(np.float32)
    data = cents + 0.01 * rng.standard_normal((K, d)).astype(np.float32)
    _check(R, oracle_mod, data, cents, Q, 40)


def test_equidistant_centroids_take_the_exact_path(R, oracle_mod):
    """3000 centroids on a sphere around the query: every approximate score
    is within the bound of the others, so the candidate list overflows and
    the exact fallback ranks them (ties by id)."""
    rng = np.random.default_rng(5)
    d, K = 64, 3000
    u = rng.standard_normal((K, d))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    center = rng.standard_normal(d).astype(np.float32) * 3
    cents = (center + 2.0 * u).astype(np.float32)
    Q = np.stack([center, center + 1e-3]).astype(np.float32)
    _check(R, oracle_mod, cents.copy(), cents, Q, 40)


@pytest.mark.parametrize("metric", ["ip", "cosine"])
def test_probe_lists_inner_product(R, oracle_mod, metric):
    rng = np.random.default_rng(9)
    d, K = 96, 777
    cents = (rng.standard_normal((K, d)) * rng.uniform(0.5, 3, (K, 1))).astype(np.float32)
    data = cents + (rng.standard_normal((K, d)) * 0.2).astype(np.float32)
    Q = (rng.standard_normal((16, d)) * 2).astype(np.float32)
    _check(R, oracle_mod, data, cents, Q, 33, metric)
