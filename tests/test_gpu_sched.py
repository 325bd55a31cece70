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
