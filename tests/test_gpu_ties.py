"""Inputs with many equal keys, against the oracle element by element.

A bucket of 700 identical points gives 700-way ties everywhere the search
ranks: equal codes and factors, so equal estimates, bounds and exact
distances. The k-th smallest upper bound, the pilot (m smallest (estimate,
id)), the survivors and the top-k are then decided by the id order of §4's
canonical (distance, id) ranking, and the selections meet key ranges of
width zero. An index whose points are all identical adds empty clusters
(k-means) and equal centroid scores in the probe selection. Every scan
form is compared: the CTA and warp layouts, bulk-copy staged rounds, the
bucket-major tensor-core scan, the split mode of small batches and a search
plan."""
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


def _same(a, b):
    return np.array_equal(np.asarray(a).view(np.uint32), np.asarray(b).view(np.uint32))


def _tied_workload(d):
    rng = np.random.default_rng(21)
    data = rng.standard_normal((4000, d)).astype(np.float32)
    data[1000:1700] = data[1000]
    Q = rng.standard_normal((40, d)).astype(np.float32)
    Q[0] = data[1000]
    Q[1] = data[1000] + np.float32(1e-3)
    Q[2] = data[1000] * np.float32(1.5)
    return data, Q


def _variants(R):
    return (dict(layout=R.LAYOUT_CTA, staging=R.STAGING_OFF),
            dict(layout=R.LAYOUT_WARP, lane_pairs=1),
            dict(layout=R.LAYOUT_WARP, lane_pairs=2),
            dict(layout=R.LAYOUT_CTA, staging=R.STAGING_BULK),
            dict(scan_path=R.SCAN_TC))


@pytest.mark.parametrize("d", [128, 200])
def test_mass_ties_match_oracle(R, oracle_mod, d):
    import torch
    data, Q = _tied_workload(d)
    G = R.Index.build(data, 24, seed=4)
    O = oracle_mod.OracleIndex(data, K=24, seed=4)
    assert _same(G.factors(), O.factors) and np.array_equal(G.assign(), O.assign)
    qd = torch.from_numpy(Q).cuda()
    for k, nprobe in ((100, 4), (10, 24), (128, 2), (1, 1)):
        ids_o, dist_o = O.search(Q, k, nprobe)
        assert (ids_o[0] == np.arange(1000, 1000 + k)).all()
        for kw in _variants(R):
            ids, dist = G.search(qd, k, nprobe, **kw)
            assert np.array_equal(ids.cpu().numpy(), ids_o), (k, nprobe, kw)
            assert _same(dist.cpu().numpy(), dist_o), (k, nprobe, kw)
        for nq in (1, 3):                      # small batches: split mode
            ids, dist = G.search(Q[:nq], k, nprobe)
            assert np.array_equal(ids, ids_o[:nq]) and _same(dist, dist_o[:nq])
    plan = R.Plan(G, 100, 4, len(Q))
    plan.queries.copy_(qd)
    plan.run(len(Q))
    plan.sync()
    ids_o, dist_o = O.search(Q, 100, 4)
    assert np.array_equal(plan.ids.cpu().numpy(), ids_o)
    assert _same(plan.dist.cpu().numpy(), dist_o)


def test_identical_points_match_oracle(R, oracle_mod):
    """All 500 points equal: one non-empty cluster, equal centroid scores,
    every distance equal; results are the lowest ids."""
    import torch
    rng = np.random.default_rng(22)
    data = np.repeat(rng.standard_normal((1, 128)).astype(np.float32), 500, axis=0)
    Q = rng.standard_normal((20, 128)).astype(np.float32)
    Q[0] = data[0]
    G = R.Index.build(data, 4, seed=4)
    O = oracle_mod.OracleIndex(data, K=4, seed=4)
    assert _same(G.centroids(), O.centroids) and np.array_equal(G.assign(), O.assign)
    assert _same(G.factors(), O.factors)
    qd = torch.from_numpy(Q).cuda()
    for k, nprobe in ((10, 4), (100, 1), (128, 2)):
        ids_o, dist_o = O.search(Q, k, nprobe)
        assert (ids_o == np.arange(k)).all()
        for kw in _variants(R):
            ids, dist = G.search(qd, k, nprobe, **kw)
            assert np.array_equal(ids.cpu().numpy(), ids_o), (k, nprobe, kw)
            assert _same(dist.cpu().numpy(), dist_o), (k, nprobe, kw)
