"""The entry point that allocates no device memory (tm_match_noalloc).

Some callers cannot allocate GPU memory while they run: a real-time receiver
loop (cudaMalloc and cudaFree can synchronise the whole device and take
unbounded time), a process whose memory already belongs to another
allocator's pool, code that may only allocate at start-up. For them the
library keeps one fixed scratch array per GPU; these tests check that a
query run through it gives what tm_match gives (exactly for +-1 signals,
within the 1e-5 / 2e-3 bars for fp32 / fp16 storage), twice in a row (the
second call reuses the array the first one left behind), for every signal
storage type and the Thm. 2 sampling, and that the second call changes the
device's free memory by nothing.

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


CASES = [
    # (queries: (seed, N, K, flip_p, t_sigma), xdtype, thm2)
    ([(71, (1 << 20) + 9, 2048, 0.05, 0.0), (72, 65536, 1024, 0.0, 0.0)], "i8", False),
    ([(73, (1 << 20) + 40, 2048, 0.05, 0.0), (74, 300000, 700, 0.02, 0.0)], "bits", False),
    ([(75, (1 << 19) + 3, 1024, 0.0, 0.3), (76, 70000, 900, 0.0, 0.3)], "f32", False),
    ([(77, (1 << 19) + 6, 1024, 0.0, 0.3), (78, 90000, 512, 0.0, 0.3)], "f16", False),
    ([(79, 200000, 1024, 0.05, 0.0), (80, 1 << 18, 600, 0.05, 0.0)], "i8", True),
]


def _close(a, b, tol):
    return abs(a - b) <= tol * max(1.0, abs(b))


@pytest.mark.gpu
@pytest.mark.parametrize("specs,xdtype,thm2", CASES, ids=["i8", "bits", "f32", "f16", "thm2"])
def test_noalloc_equals_tm_match_twice(tm, specs, xdtype, thm2):
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    tol = 2e-3 if xdtype == "f16" else 1e-5
    for k, (seed, N, K, flip_p, t_sigma) in enumerate(specs):
        q = W.planted_query(seed, N, K, xdtype, flip_p=flip_p, t_sigma=t_sigma, mode="auto")
        x = torch.from_numpy(q.x).cuda()
        t = torch.from_numpy(q.t).cuda()
        ref = tm.result_buffer(1)
        p = tm.Plan(q.N, q.K, xdtype, "auto", thm2=thm2)
        p.match(x, t, ref)
        got = tm.result_buffer(1)
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        tm.tm_match_noalloc(x, t, got, N=q.N, K=q.K, xdtype=xdtype, mode="auto", thm2=thm2)
        torch.cuda.synchronize()
        if k == 1:   # the second call in a row: set-up done, nothing allocated
            assert torch.cuda.mem_get_info()[0] == free0
        r_ref = tm.decode_results(ref)[0]
        r_got = tm.decode_results(got)[0]
        if xdtype in ("i8", "bits"):
            # integer signal, integer template: every field is exact
            assert r_got == r_ref, (r_got, r_ref)
        else:
            # real signals: the fold's fp32 sums may be grouped differently
            # (the array holds fewer partial shares), so values agree within
            # the storage type's bar; the planted peaks here are far from ties
            for key in ("shift", "status", "n_cand", "m1", "m2"):
                assert r_got[key] == r_ref[key], (key, r_got, r_ref)
            for key in ("r1", "r2", "score"):
                assert _close(r_got[key], r_ref[key], tol), (key, r_got[key], r_ref[key])
        p.close()


@pytest.mark.gpu
def test_noalloc_captured_in_a_graph(tm):
    """A call captured into a CUDA graph (after a first call outside any
    capture) replays correctly: its descriptors travel as kernel
    parameters, so the graph holds no pointer to a host stack frame.
    Replaying after the captured buffers are refilled with another query
    of the same shape gives that query's result."""
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    N, K = (1 << 20) + 16, 2048   # a fold with 16 rows of shares: the slot sums are captured too
    qa = W.planted_query(81, N, K, "i8", flip_p=0.05, mode="auto")
    qb = W.planted_query(82, N, K, "i8", flip_p=0.05, mode="auto")
    x = torch.from_numpy(qa.x).cuda()
    t = torch.from_numpy(qa.t).cuda()
    out = tm.result_buffer(1)
    tm.tm_match_noalloc(x, t, out, N=N, K=K, xdtype="i8", mode="auto")   # first call: set-up outside capture
    torch.cuda.synchronize()
    want_a = tm.decode_results(out)[0]
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        tm.tm_match_noalloc(x, t, out, N=N, K=K, xdtype="i8", mode="auto", stream=s)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert tm.decode_results(out)[0] == want_a
    # the same graph on another query's data in the captured buffers
    ref_b = tm.result_buffer(1)
    xb = torch.from_numpy(qb.x).cuda()
    tb = torch.from_numpy(qb.t).cuda()
    tm.tm_match_noalloc(xb, tb, ref_b, N=N, K=K, xdtype="i8", mode="auto")
    torch.cuda.synchronize()
    x.copy_(xb)
    t.copy_(tb)
    out.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert tm.decode_results(out)[0] == tm.decode_results(ref_b)[0]
