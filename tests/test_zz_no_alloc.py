"""rabitq_search_noalloc, called through the C-ABI, returns what rabitq_search
returns, on two calls in a row (the calls share the library's fixed scratch
array, so the second call also checks that leftovers of the first do not leak
into its results).

This file is named to be collected last: the entry point is for callers that
cannot allocate device memory when they search (their allocator already owns
the GPU's memory, or the path must not pay an allocation), and it must work
whether or not other tests ran before it in the same process.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(R, G, qd, k, nprobe, bq=4, eps0=1.9, npq=None):
    import torch
    nq = qd.shape[0]
    ids = torch.full((nq, k), -7, dtype=torch.int64, device=qd.device)
    dist = torch.full((nq, k), float("nan"), dtype=torch.float32, device=qd.device)
    o = R.SearchOpts()
    R.lib().rabitq_search_opts_default(C.byref(o))
    o.io_on_device = 1
    o.stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if npq is not None:  # a device int32 tensor of nq probe counts
        o.per_query_nprobe = C.c_void_p(npq.data_ptr())
    rc = R.lib().rabitq_search_noalloc(G._h, C.c_void_p(qd.data_ptr()), nq, k, nprobe, bq, eps0,
                                       C.c_void_p(ids.data_ptr()), C.c_void_p(dist.data_ptr()),
                                       C.byref(o))
    torch.cuda.synchronize()
    return rc, ids.cpu().numpy(), dist.cpu().numpy()


@pytest.mark.parametrize("case", ["tiny", "chunked"])
def test_noalloc_matches_search_on_two_calls(case):
    import torch
    from paper_2405_12497_gb300 import build, rabitq as R, synth
    assert torch.cuda.is_available()
    build.build()
    if case == "tiny":
        data, Q = synth.tiny()
        G = R.Index.build(data, 16, seed=2)
        k, nprobe = 10, 4
    else:  # several query chunks through the fixed scratch
        data, Q = synth.sift_like(200_000, 5000)
        G = R.Index.build(data, 4096, seed=2)
        k, nprobe = 100, 16
    qd = torch.from_numpy(Q).cuda()
    ref_ids, ref_dist = G.search(qd, k, nprobe)
    ref_ids, ref_dist = ref_ids.cpu().numpy(), ref_dist.cpu().numpy()
    for _ in range(2):
        rc, ids, dist = _noalloc(R, G, qd, k, nprobe)
        assert rc == R.OK, R.lib().rabitq_last_error()
        assert np.array_equal(ids, ref_ids)
        assert np.array_equal(dist.view(np.uint32), ref_dist.view(np.uint32))


def test_noalloc_rejects_host_buffers():
    import torch
    from paper_2405_12497_gb300 import build, rabitq as R, synth
    build.build()
    data, Q = synth.tiny(n=2000, nq=4)
    G = R.Index.build(data, 8, seed=2)
    ids = np.zeros((4, 5), np.int64)
    dist = np.zeros((4, 5), np.float32)
    rc = R.lib().rabitq_search_noalloc(G._h, Q.ctypes.data_as(C.c_void_p), 4, 5, 2, 4, 1.9,
                                       ids.ctypes.data_as(C.c_void_p),
                                       dist.ctypes.data_as(C.c_void_p), None)
    assert rc == R.EINVAL
    assert b"device memory" in R.lib().rabitq_last_error()


def test_noalloc_reports_non_finite_query():
    """A NaN or infinite query value is an EINVAL, as for rabitq_search; a
    clean call right after it succeeds (the flag starts at zero each call)."""
    import torch
    from paper_2405_12497_gb300 import build, rabitq as R, synth
    build.build()
    data, Q = synth.tiny(n=2000, nq=8)
    G = R.Index.build(data, 8, seed=2)
    for bad in (float("nan"), float("inf")):
        Qb = Q.copy()
        Qb[3, 17] = bad
        rc, _, _ = _noalloc(R, G, torch.from_numpy(Qb).cuda(), 5, 2)
        assert rc == R.EINVAL
        assert b"non-finite" in R.lib().rabitq_last_error()
    qd = torch.from_numpy(Q).cuda()
    rc, ids, dist = _noalloc(R, G, qd, 5, 2)
    assert rc == R.OK, R.lib().rabitq_last_error()
    ref_ids, ref_dist = G.search(qd, 5, 2)
    assert np.array_equal(ids, ref_ids.cpu().numpy())
    assert np.array_equal(dist.view(np.uint32), ref_dist.cpu().numpy().view(np.uint32))


def test_noalloc_matches_oracle(oracle_mod):
    """Against the oracle directly: every metric, the largest k (1024) and
    per-query probe counts, through the fixed scratch."""
    import torch
    from paper_2405_12497_gb300 import build, rabitq as R, synth
    build.build()
    data, Q = synth.tiny()
    Q = Q[:40]
    qd = torch.from_numpy(Q).cuda()
    for metric in ("l2", "ip", "cosine"):
        G = R.Index.build(data, 16, seed=2, metric=metric)
        O = oracle_mod.OracleIndex(data, K=16, seed=2, metric=metric)
        for k, nprobe in ((10, 4), (1024, 16)):
            rc, ids, dist = _noalloc(R, G, qd, k, nprobe)
            assert rc == R.OK, R.lib().rabitq_last_error()
            ids_o, dist_o = O.search(Q, k, nprobe)
            assert np.array_equal(ids, ids_o), (metric, k)
            assert np.array_equal(dist.view(np.uint32), dist_o.view(np.uint32)), (metric, k)
        if metric == "l2":
            npq = ((np.arange(len(Q)) * 7) % 9 + 1).astype(np.int32)
            rc, ids, dist = _noalloc(R, G, qd, 10, 9, npq=torch.from_numpy(npq).cuda())
            assert rc == R.OK, R.lib().rabitq_last_error()
            ids_o, dist_o = O.search(Q, 10, 9, per_query_nprobe=npq)
            assert np.array_equal(ids, ids_o)
            assert np.array_equal(dist.view(np.uint32), dist_o.view(np.uint32))
        G.free()
