"""Scan-path autotuner (and the scheduling around the search) on the GPU."""
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


def test_autotune_picks_a_path_and_auto_follows_it(R, tiny_workload):
    data, queries = tiny_workload
    idx = R.Index.build(data, 16, seed=2, kmeans_iters=10)
    chosen, t = idx.autotune(queries, 10, 4, reps=2)
    assert chosen in (R.SCAN_POPC, R.SCAN_TC)
    assert t["popc"] > 0 and (t["tc"] > 0 or t["tc"] == -1)
    if t["tc"] > 0:
        assert chosen == (R.SCAN_TC if t["tc"] < t["popc"] else R.SCAN_POPC)
    a = idx.search(queries, 10, 4)                       # AUTO
    b = idx.search(queries, 10, 4, scan_path=R.SCAN_POPC)
    c = idx.search(queries, 10, 4, scan_path=R.SCAN_TC)
    for x in (b, c):
        assert np.array_equal(a[0], x[0])
        assert np.array_equal(a[1].view(np.uint32), x[1].view(np.uint32))


def test_autotune_rejects_bad_arguments(R, tiny_workload):
    data, queries = tiny_workload
    idx = R.Index.build(data, 16, seed=2, kmeans_iters=2)
    with pytest.raises(R.RabitqError):
        idx.autotune(queries, 10, 4, reps=0)
    with pytest.raises(R.RabitqError):
        idx.autotune(queries, 10, 99)                    # nprobe > K


@pytest.fixture(scope="module")
def tiny_idx(R, tiny_workload):
    data, _ = tiny_workload
    return R.Index.build(data, 16, seed=2, kmeans_iters=10)


def _same(a, b):
    assert np.array_equal(np.asarray(a[0]), np.asarray(b[0]))
    assert np.array_equal(np.asarray(a[1]).view(np.uint32), np.asarray(b[1]).view(np.uint32))


@pytest.mark.parametrize("rot", ["fp32", "bf16"])
def test_plan_replays_equal_search(R, tiny_workload, tiny_idx, rot):
    import torch
    _, queries = tiny_workload
    rp = R.ROT_FP32 if rot == "fp32" else R.ROT_BF16
    plan = R.Plan(tiny_idx, 10, 5, 100, rot_precision=rp)
    qd = torch.from_numpy(queries).cuda()
    for nq in (100, 1, 37, 100, 37):           # new sizes capture, repeats replay
        plan.queries[:nq].copy_(qd[:nq])
        plan.run(nq)
        plan.sync()
        ref = tiny_idx.search(queries[:nq], 10, 5, scan_path=R.SCAN_POPC, rot_precision=rp)
        _same((plan.ids[:nq].cpu().numpy(), plan.dist[:nq].cpu().numpy()), ref)
    # round trip through host memory
    _same(plan.search(queries[:50]), tiny_idx.search(queries[:50], 10, 5, scan_path=R.SCAN_POPC,
                                                      rot_precision=rp))
    with pytest.raises(R.RabitqError):
        plan.run(101)                           # more than nq_max


def test_plan_with_predictor_equals_learned_search(R, tiny_workload, tiny_idx):
    import math
    _, queries = tiny_workload
    rng = np.random.default_rng(3)
    from oracle import mlp_oracle as M
    p = M.pack(rng.uniform(-1, 1, (64, 256)) * math.sqrt(6 / 64), rng.normal(0, .1, 256),
               rng.uniform(-1, 1, (256, 256)) * math.sqrt(6 / 256), rng.normal(0, .1, 256),
               rng.uniform(-1, 1, 256) * math.sqrt(6 / 256), 2.0).astype(np.float32)
    for nmax in (12, 16):
        pr = R.Predictor.create(p, 30.0, 1.0, nmax, 16)
        plan = R.Plan(tiny_idx, 10, 0, 100, predictor=pr)
        _same(plan.search(queries), tiny_idx.search_learned(pr, queries, 10,
                                                            scan_path=R.SCAN_POPC))
        assert np.array_equal(plan.nprobe.cpu().numpy(), tiny_idx.predict_nprobe(pr, queries))


def test_plan_reports_overflow_like_search(R, tiny_workload, tiny_idx):
    _, queries = tiny_workload
    try:
        ref = tiny_idx.search(queries, 100, 16, max_candidates=4096, scan_path=R.SCAN_POPC)
        ref_err = None
    except R.RabitqError as e:
        ref, ref_err = None, e.code
    plan = R.Plan(tiny_idx, 100, 16, 100, max_candidates=4096)
    if ref_err is None:
        _same(plan.search(queries), ref)
    else:
        with pytest.raises(R.RabitqError) as ei:
            plan.search(queries)
        assert ei.value.code == ref_err
        # the sync that reported the error cleared the flag
        plan.sync()


def test_min_candidate_capacity(R, tiny_workload, tiny_idx):
    _, queries = tiny_workload
    with pytest.raises(R.RabitqError):
        tiny_idx.search(queries, 10, 4, max_candidates=4095)
    with pytest.raises(R.RabitqError):
        R.Plan(tiny_idx, 10, 4, 100, max_candidates=4095)
    _same(tiny_idx.search(queries, 10, 2, max_candidates=4096),
          tiny_idx.search(queries, 10, 2))


def test_plan_rejects_bad_arguments(R, tiny_idx):
    with pytest.raises(R.RabitqError):
        R.Plan(tiny_idx, 10, 17, 100)            # nprobe > K
    with pytest.raises(R.RabitqError):
        R.Plan(tiny_idx, 0, 4, 100)              # k < 1
    with pytest.raises(R.RabitqError):
        R.Plan(tiny_idx, 10, 4, 0)               # nq_max < 1


def test_split_batches_equal_unsplit(R, tiny_workload, tiny_idx):
    """Small batches split each query's probes over several CTAs and merge
    them; the results equal those of a batch large enough not to split."""
    _, queries = tiny_workload
    big = np.concatenate([queries] * 6)            # 600 queries: no split
    ref_ids, ref_dist = tiny_idx.search(big, 10, 8, scan_path=R.SCAN_POPC)
    for nq in (1, 3, 50):
        ids, dist = tiny_idx.search(queries[:nq], 10, 8, scan_path=R.SCAN_POPC)
        assert np.array_equal(ids, ref_ids[:nq])
        assert np.array_equal(dist.view(np.uint32), ref_dist[:nq].view(np.uint32))
    # through a plan (CUDA graph) as well, k = 100 and every probe
    ref_ids, ref_dist = tiny_idx.search(big, 100, 16, scan_path=R.SCAN_POPC)
    plan = R.Plan(tiny_idx, 100, 16, 64)
    for nq in (1, 7, 64):
        ids, dist = plan.search(queries[:nq])
        assert np.array_equal(ids, ref_ids[:nq])
        assert np.array_equal(dist.view(np.uint32), ref_dist[:nq].view(np.uint32))


def test_tile_autotuner_times_every_tile_and_auto_follows(R, tiny_workload):
    """rabitq_autotune_tiles times every work decomposition of the scan
    (CTA per query; warp per query with 1 or 2 codes per lane per step; the
    tensor-core path), caches the fastest for the shape class, and AUTO
    searches and new plans take it; every tile returns the oracle's bits."""
    import torch
    from oracle import oracle as O
    O.build()
    data, queries = tiny_workload
    idx = R.Index.build(data, 16, seed=2, kmeans_iters=10)
    best, every = idx.autotune_tiles(queries, 10, 4, reps=2)
    kinds = {(t["scan_path"], t["layout"], t["lane_pairs"]) for t in every}
    assert ("popcount", "cta-per-query", 0) in kinds
    assert ("popcount", "warp-per-query", 1) in kinds and ("popcount", "warp-per-query", 2) in kinds
    ok = [t for t in every if t["time_ms"] > 0]
    assert best["time_ms"] == min(t["time_ms"] for t in ok)
    ids_o, dist_o = O.OracleIndex(data, K=16, seed=2).search(queries, 10, 4)
    qd = torch.from_numpy(queries).cuda()
    for path, lay, lp in ((R.SCAN_POPC, R.LAYOUT_CTA, 0), (R.SCAN_POPC, R.LAYOUT_WARP, 1),
                          (R.SCAN_POPC, R.LAYOUT_WARP, 2), (R.SCAN_TC, R.LAYOUT_AUTO, 0),
                          (R.SCAN_AUTO, R.LAYOUT_AUTO, 0)):
        ids, dist = idx.search(qd, 10, 4, scan_path=path, layout=lay, lane_pairs=lp)
        assert np.array_equal(ids.cpu().numpy(), ids_o)
        assert np.array_equal(dist.cpu().numpy().view(np.uint32), dist_o.view(np.uint32))
    plan = R.Plan(idx, 10, 4, 100)
    if best["scan_path"] == "popcount":
        t = plan.tile()
        assert t["layout"] == best["layout"] and t["lane_pairs"] == best["lane_pairs"]
    plan.queries.copy_(qd)
    plan.run(100)
    plan.sync()
    assert np.array_equal(plan.ids.cpu().numpy(), ids_o)


def test_tile_options_are_checked(R, tiny_idx, tiny_workload):
    _, queries = tiny_workload
    with pytest.raises(R.RabitqError):
        tiny_idx.search(queries, 10, 4, lane_pairs=3)
    with pytest.raises(R.RabitqError):
        tiny_idx.search(queries, 10, 4, layout=7)


def test_search_stats_and_their_error_path(R, tiny_workload, tiny_idx):
    """Stage times recorded with stats on leave the results unchanged, on
    both scan paths; a non-finite query with stats on is EINVAL and the
    next searches (with their timing events) still run."""
    _, queries = tiny_workload
    for path in (R.SCAN_POPC, R.SCAN_TC):
        want = tiny_idx.search(queries, 10, 4, scan_path=path)
        got = tiny_idx.search(queries, 10, 4, scan_path=path, stats=True)
        _same(got, want)
        st = R.last_stats()
        assert len(st) == 5 and (st >= 0).all() and st[4] > 0
    bad = queries[:5].copy()
    bad[1, 3] = np.inf
    for _ in range(50):
        with pytest.raises(R.RabitqError) as e:
            tiny_idx.search(bad, 10, 4, stats=True)
        assert e.value.code == R.EINVAL
    _same(tiny_idx.search(queries, 10, 4, stats=True), tiny_idx.search(queries, 10, 4))
