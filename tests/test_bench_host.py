"""The benchmark's host-side pieces on CPU: the ground truth its recall is
measured against (exact kNN / maximum inner product, candidates by an FP32
product then FP64 refinement) equals brute force, and recall@k counts set
overlap."""
import numpy as np
import torch


def test_exact_knn_equals_brute_force(oracle_mod, tiny_workload):
    import bench
    data, Q = tiny_workload
    gt = bench.exact_knn(torch.from_numpy(data), torch.from_numpy(Q), 10)
    d64 = ((Q.astype(np.float64)[:, None, :] - data[None].astype(np.float64)) ** 2).sum(-1)
    want = np.argsort(d64, axis=1, kind="stable")[:, :10]
    same = (gt == want).all(1)
    assert same.mean() >= 0.99      # an exact FP64 tie may order differently
    # where they differ, the returned set has the same distances
    for i in np.where(~same)[0]:
        assert np.allclose(np.sort(d64[i, gt[i]]), np.sort(d64[i, want[i]]))
    ids, _ = oracle_mod.bruteforce_knn(data, Q, 10)
    assert bench.recall_at(ids, gt) >= 0.999


def test_exact_mips_and_cosine_equal_brute_force(tiny_workload):
    import bench
    data, Q = tiny_workload
    gt = bench.exact_mips(torch.from_numpy(data), torch.from_numpy(Q), 10)
    ip = Q.astype(np.float64) @ data.astype(np.float64).T
    want = np.argsort(-ip, axis=1, kind="stable")[:, :10]
    assert bench.recall_at(gt, want) >= 0.999
    gc = bench.exact_mips(torch.from_numpy(data), torch.from_numpy(Q), 10, cosine=True)
    cos = ip / np.linalg.norm(data.astype(np.float64), axis=1)[None]
    wc = np.argsort(-cos, axis=1, kind="stable")[:, :10]
    assert bench.recall_at(gc, wc) >= 0.999


def test_recall_counts_overlap():
    import bench
    gt = np.array([[1, 2, 3, 4], [5, 6, 7, 8]])
    ids = np.array([[4, 3, 9, 9, 1], [0, 0, 0, 0, 5]])
    assert bench.recall_at(ids, gt) == (2 / 4 + 0 / 4) / 2   # only the first k ids count


def test_clock_summary_keeps_the_timed_region_and_flags_throttling():
    import bench
    s = bench.ClockSampler(0)
    row = "0, {sm}, 2070, 900.00, 0x0000000000000000, {hw}, Not Active, Not Active, {pc}"
    s.lines = [(0.5, row.format(sm=1200, hw="Not Active", pc="Not Active")),   # before
               (1.1, row.format(sm=2070, hw="Not Active", pc="Active")),
               (1.2, row.format(sm=1965, hw="Not Active", pc="Not Active")),
               (1.3, row.format(sm=2070, hw="Not Active", pc="Not Active")),
               (2.5, row.format(sm=900, hw="Active", pc="Not Active"))]      # after
    s.t0, s.t1 = 1.0, 1.35
    out = s.summary()
    assert out["samples"] == 3 and out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"]
    s.t0, s.t1 = 2.0, 2.1          # a region shorter than a period: the next sample
    out = s.summary()
    assert out["samples"] == 1 and out["reasons"] == ["hw_slowdown"]
    s.lines = []
    assert s.summary()["reasons"] == ["unsampled"]
