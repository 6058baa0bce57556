"""Failure detection on the GPU without a fault: a bounded device-side wait
on a barrier that nothing arrives at gives up at its limit and reports it,
the call returns promptly, and the context stays usable afterwards."""
import time

import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tm():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1509_04863_gb300 import _build
    _build.build()
    import paper_1509_04863_gb300 as tm
    return tm


def test_bounded_wait_gives_up_and_context_survives(tm):
    t0 = time.perf_counter()
    assert tm.selftest_wait_timeout(2_000_000)   # 2 ms limit
    assert time.perf_counter() - t0 < 5.0
    # the device still runs work normally
    q = W.planted_query(3, 65536, 1024, "i8", mode="paper")
    b = tm.Batch([dict(x=torch.from_numpy(q.x).cuda(), t=torch.from_numpy(q.t).cuda(), N=q.N, K=q.K,
                       xdtype="i8", mode="paper")])
    out = tm.result_buffer(1)
    b.run(out)
    torch.cuda.synchronize()
    assert b.device_error() == 0
    assert tm.decode_results(out)[0]["status"] & 0xFF in (0, 1, 2)
