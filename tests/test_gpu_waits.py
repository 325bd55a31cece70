"""The bounded mbarrier waits of the tensor-core kernels give up instead of
hanging: a kernel waits on a barrier nothing completes (it must stop after
its poll limit) and on one while another warp raises the CTA's failure flag
(it must stop on the flag); the kernel returns, the error is reported to
the host, and the context keeps working (a search afterwards matches the
oracle)."""
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


@pytest.mark.parametrize("polls", [1, 1 << 12, 1 << 16])
def test_bounded_waits_give_up(R, polls):
    R.selftest_wait(polls)


def test_zero_polls_is_einval(R):
    with pytest.raises(R.RabitqError) as e:
        R.selftest_wait(0)
    assert e.value.code == R.EINVAL


def test_context_usable_after_timeouts(R, oracle_mod, tiny_workload):
    data, Q = tiny_workload
    R.selftest_wait(1 << 10)
    G = R.Index.build(data, 16, seed=2)
    O = oracle_mod.OracleIndex(data, K=16, seed=2)
    ids, dist = G.search(Q[:20], 10, 4)
    ids_o, dist_o = O.search(Q[:20], 10, 4)
    assert np.array_equal(ids, ids_o)
    assert np.array_equal(dist.view(np.uint32), dist_o.view(np.uint32))
