"""The entry point that allocates no device memory (tm_match_noalloc).

Some callers cannot allocate GPU memory while they run: a real-time receiver
loop (cudaMalloc and cudaFree can synchronise the whole device and take
unbounded time), a process whose memory already belongs to another
allocator's pool, code that may only allocate at start-up. For them the
library keeps one fixed scratch array per GPU; these tests check that a
query run through it gives exactly what tm_match gives, twice in a row (the
second call reuses the array the first one left behind).

This file is named to be collected last.
"""
import pytest
import torch

import workloads as W


@pytest.fixture(scope="module")
def tm():
    from paper_1509_04863_gb300 import _build
    _build.build()
    import paper_1509_04863_gb300 as tm
    return tm


def test_noalloc_rejects_what_does_not_fit(tm):
    """A signal above TM_NOALLOC_MAX_SIGNAL_BYTES (256 MiB) is refused with a
    clear error before any GPU work (no device needed)."""
    x = torch.zeros(16, dtype=torch.int8)   # never read: the size check comes first
    with pytest.raises(tm.TMError) as e:
        tm.tm_match_noalloc(x, torch.zeros(4, dtype=torch.float32), torch.zeros(tm.RESULT_BYTES // 8, dtype=torch.int64),
                            N=(1 << 28) + 16, K=4096, mode="paper", allow_ambig=True)
    assert e.value.status == tm.TM_EUNSUPPORTED
    assert "no-allocation" in str(e.value)


@pytest.mark.gpu
def test_noalloc_equals_tm_match_twice(tm):
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    queries = [W.planted_query(71, (1 << 20) + 9, 2048, "i8", flip_p=0.05),
               W.planted_query(72, 65536, 1024, "i8", flip_p=0.0)]
    for q in queries:
        x = torch.from_numpy(q.x).cuda()
        t = torch.from_numpy(q.t).cuda()
        ref = tm.result_buffer(1)
        p = tm.Plan(q.N, q.K, "i8", "paper")
        p.match(x, t, ref)
        got = tm.result_buffer(1)
        tm.tm_match_noalloc(x, t, got, N=q.N, K=q.K, xdtype="i8", mode="paper")
        torch.cuda.synchronize()
        r_ref = tm.decode_results(ref)[0]
        r_got = tm.decode_results(got)[0]
        # integer signal, integer template: every field is exact
        assert r_got == r_ref, (r_got, r_ref)
        p.close()
