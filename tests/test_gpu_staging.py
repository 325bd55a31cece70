"""Bulk-copy staging of the CTA layout's scan rounds (RABITQ_STAGING_BULK:
each round's codes and factors are copied into shared memory by the bulk-copy
engine while the block evaluates the round before) against the oracle and
against the unstaged kernel, element by element: both code lengths it
covers (D' = 128, 256), rounds that span dozens of small or empty buckets,
the split mode, the inner-product metric, and a candidate overflow that
ends a round early (the copies in flight are waited for; the next search is
unaffected)."""
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


def _check(R, G, O, Q, k, nprobe, eps0=1.9, **kw):
    import torch
    qd = torch.from_numpy(Q).cuda()
    ids_o, dist_o = O.search(Q, k, nprobe, eps0=eps0)
    for st in (R.STAGING_BULK, R.STAGING_OFF):
        ids, dist = G.search(qd, k, nprobe, eps0=eps0, layout=R.LAYOUT_CTA, staging=st, **kw)
        assert np.array_equal(ids.cpu().numpy(), ids_o), st
        assert _same(dist.cpu().numpy(), dist_o), st


@pytest.fixture(scope="module")
def tiny(R, oracle_mod, tiny_workload):
    data, Q = tiny_workload
    return R.Index.build(data, 16, seed=2), oracle_mod.OracleIndex(data, K=16, seed=2), Q


@pytest.mark.parametrize("k,nprobe,eps0", [(10, 4, 1.9), (100, 16, 1.9), (1, 1, 0.0), (50, 7, 3.0)])
def test_staged_d128_matches_oracle(R, tiny, k, nprobe, eps0):
    G, O, Q = tiny
    _check(R, G, O, Q, k, nprobe, eps0)


def test_staged_d256_matches_oracle(R, oracle_mod):
    from paper_2405_12497_gb300 import synth
    data, Q = synth.tiny(n=6000, d=200, nq=60)
    G = R.Index.build(data, 24, seed=2)
    O = oracle_mod.OracleIndex(data, K=24, seed=2)
    for k, nprobe in ((10, 3), (100, 12)):
        _check(R, G, O, Q, k, nprobe)


def test_staged_rounds_over_many_small_buckets(R, oracle_mod):
    """3000 points in 1000 buckets: a 256-pair round spans dozens of bucket
    runs, more than one per lane of the issuing warp."""
    from paper_2405_12497_gb300 import synth
    data, Q = synth.tiny(n=3000, nq=40)
    G = R.Index.build(data, 1000, seed=2, kmeans_iters=3)
    O = oracle_mod.OracleIndex(data, K=1000, seed=2, iters=3)
    off, _ = G.buckets()
    assert np.diff(off).mean() < 4      # a round of 256 pairs spans over 64 buckets
    _check(R, G, O, Q, 10, 300)
    _check(R, G, O, Q, 100, 1000)


def test_staged_split_mode_and_inner_product(R, oracle_mod, tiny, tiny_workload):
    G, O, Q = tiny
    _check(R, G, O, Q[:2], 10, 16)             # two queries: split over CTAs
    data, _ = tiny_workload
    Gi = R.Index.build(data, 16, seed=2, metric="ip")
    Oi = oracle_mod.OracleIndex(data, K=16, seed=2, metric="ip")
    _check(R, Gi, Oi, Q[:50], 20, 5)


def test_staged_overflow_is_reported_and_harmless(R, tiny):
    """Every bucket probed with a very wide bound: more than 4096 candidates,
    a round ends the scan early with the next round's copies in flight; the
    search reports the overflow, and the next search is exact."""
    import torch
    G, O, Q = tiny
    qd = torch.from_numpy(np.concatenate([Q] * 5)).cuda()   # 500 queries: no split
    with pytest.raises(R.RabitqError) as e:
        G.search(qd, 10, 16, eps0=50.0, max_candidates=4096, layout=R.LAYOUT_CTA,
                 staging=R.STAGING_BULK)
    assert e.value.code == -7
    _check(R, G, O, Q[:8], 10, 4)
