"""The warp-per-query layout of the fused scan (one warp per query, no block
barrier; RABITQ_LAYOUT_WARP) against the oracle, element by element: the
same probe lists, quantization stream, estimator, error-bound pruning and
re-ranking rule (§4), so ids and distance bits are identical. Covered: both
code lengths it handles (D' = 128 and 256), k from 1 to its maximum of 128,
fewer than k codes in the probed buckets (padding), inner products and
cosines, per-query probe counts, candidate lists that outgrow a warp's
region (handed back to the CTA kernel), parameters outside its range (the
CTA kernel runs) and a search plan (CUDA graph)."""
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


def _check(R, G, O, Q, k, nprobe, eps0=1.9, bq=4, **kw):
    import torch
    qd = torch.from_numpy(Q).cuda()
    ids_w, dist_w = G.search(qd, k, nprobe, bq=bq, eps0=eps0, layout=R.LAYOUT_WARP, **kw)
    ids_c, dist_c = G.search(qd, k, nprobe, bq=bq, eps0=eps0, layout=R.LAYOUT_CTA, **kw)
    ids_o, dist_o = O.search(Q, k, nprobe, bq=bq, eps0=eps0)
    ids_w, dist_w = ids_w.cpu().numpy(), dist_w.cpu().numpy()
    assert np.array_equal(ids_w, ids_o)
    assert _same(dist_w, dist_o)
    assert np.array_equal(ids_c.cpu().numpy(), ids_o)
    assert _same(dist_c.cpu().numpy(), dist_o)


@pytest.fixture(scope="module")
def tiny(R, oracle_mod, tiny_workload):
    data, Q = tiny_workload
    return R.Index.build(data, 16, seed=2), oracle_mod.OracleIndex(data, K=16, seed=2), Q


@pytest.mark.parametrize("k,nprobe,eps0", [(10, 4, 1.9), (1, 1, 1.9), (128, 6, 1.9),
                                           (100, 16, 0.0), (37, 3, 3.0)])
def test_warp_layout_d128_matches_oracle(R, tiny, k, nprobe, eps0):
    G, O, Q = tiny
    _check(R, G, O, Q, k, nprobe, eps0)


def test_warp_layout_d256_matches_oracle(R, oracle_mod):
    from paper_2405_12497_gb300 import synth
    data, Q = synth.tiny(n=6000, d=200, nq=80)      # codes padded to 256 bits
    G = R.Index.build(data, 24, seed=2)
    O = oracle_mod.OracleIndex(data, K=24, seed=2)
    assert G.dpad == 256
    for k, nprobe in ((10, 4), (100, 9), (128, 24)):
        _check(R, G, O, Q, k, nprobe)


def test_warp_layout_pads_short_lists(R, oracle_mod):
    """Fewer than k codes in the probed buckets: -1 / +inf padding."""
    from paper_2405_12497_gb300 import synth
    data, Q = synth.tiny(n=2000, nq=40)
    G = R.Index.build(data, 64, seed=2)
    O = oracle_mod.OracleIndex(data, K=64, seed=2)
    _check(R, G, O, Q, 128, 2)
    import torch
    ids, dist = G.search(torch.from_numpy(Q).cuda(), 128, 2, layout=R.LAYOUT_WARP)
    assert (ids.cpu().numpy() == -1).any()


@pytest.mark.parametrize("metric", ["ip", "cosine"])
def test_warp_layout_inner_products(R, oracle_mod, tiny_workload, metric):
    data, Q = tiny_workload
    G = R.Index.build(data, 16, seed=2, metric=metric)
    O = oracle_mod.OracleIndex(data, K=16, seed=2, metric=metric)
    _check(R, G, O, Q[:60], 20, 5)


def test_warp_layout_per_query_counts(R, tiny):
    import torch
    G, O, Q = tiny
    npq = ((np.arange(len(Q)) * 7) % 9 + 1).astype(np.int32)
    qd = torch.from_numpy(Q).cuda()
    ids, dist = G.search(qd, 10, 9, per_query_nprobe=torch.from_numpy(npq).cuda(),
                         layout=R.LAYOUT_WARP)
    ids_o, dist_o = O.search(Q, 10, 9, per_query_nprobe=npq)
    assert np.array_equal(ids.cpu().numpy(), ids_o)
    assert _same(dist.cpu().numpy(), dist_o)


def test_warp_layout_hands_long_lists_to_the_cta_kernel(R, tiny):
    """With every bucket probed and a wide bound, nearly every code passes
    LB <= tau: the lists exceed a warp's 8192-entry region (the CTA kernel,
    with its 65536-entry lists, redoes those queries); results unchanged."""
    G, O, Q = tiny
    _check(R, G, O, Q[:24], 10, 16, eps0=12.0)


def test_warp_layout_outside_its_range_runs_cta(R, oracle_mod, tiny):
    """k > 128 and B_q != 4 are not in the warp kernel's range: the search
    runs in the CTA layout and still matches the oracle."""
    G, O, Q = tiny
    _check(R, G, O, Q[:30], 200, 4)
    _check(R, G, O, Q[:30], 10, 4, bq=3)


def test_warp_layout_plan_matches_oracle(R, tiny):
    import torch
    G, O, Q = tiny
    plan = R.Plan(G, 10, 4, len(Q), layout=R.LAYOUT_WARP)
    plan.queries.copy_(torch.from_numpy(Q).cuda())
    for _ in range(2):
        plan.run(len(Q))
        plan.sync()
    ids_o, dist_o = O.search(Q, 10, 4)
    assert np.array_equal(plan.ids.cpu().numpy(), ids_o)
    assert _same(plan.dist.cpu().numpy(), dist_o)
