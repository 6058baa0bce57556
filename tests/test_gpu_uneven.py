"""The uneven batch (4096 queries, N log-uniform, K log-uniform, half +-1
int8 and half N(0,1) fp32 signals with noisy templates, automatic moduli)
run as one CUDA graph.

- the graph replays give results identical to a plain tm_batch_run
  (every query, every field), replay after replay;
- a seeded sample of queries equals the oracle: bit-exact folds, maxima
  and shifts for +-1 signals, the fp32 tolerance rules for real ones;
- the same queries sharing the batch with 4095 others give the same result
  as alone, bit for bit (real signals included);
- pipelined runs on a split of the SMs, and other fold grids, give the
  same results as the plain run.

Signal lengths here span [2^14, 2^18] so the host generates the batch in
seconds; the length distribution's upper end is exercised by the other
GPU tests (N = 2^24).
"""
import numpy as np
import pytest
import torch

import oracle.ftm as O
import workloads as W
from parity import check_int, check_real, check_result

pytestmark = pytest.mark.gpu

NQ = 4096


@pytest.fixture(scope="module")
def tm():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1509_04863_gb300 import _build
    _build.build()
    import paper_1509_04863_gb300 as tm
    return tm


@pytest.fixture(scope="module")
def uneven(tm):
    qs = W.uneven(seed=5000, n=NQ, logN=(14.0, 18.0))
    specs = [dict(x=torch.from_numpy(q.x).cuda(), t=torch.from_numpy(q.t).cuda(), N=q.N, K=q.K,
                  xdtype=q.xdtype, mode=q.mode) for q in qs]
    b = tm.Batch(specs, keep_corr=True)
    return qs, specs, b


def test_graph_replays_equal_plain_run(tm, uneven):
    qs, _, b = uneven
    plain = tm.result_buffer(NQ)
    b.run(plain)
    torch.cuda.synchronize()
    want = tm.decode_results(plain)
    assert b.device_error() == 0
    out = tm.result_buffer(NQ)
    b.capture_graph(out)
    for _ in range(3):
        out.zero_()
        b.launch_graph()
        torch.cuda.synchronize()
        assert tm.decode_results(out) == want
    assert b.device_error() == 0
    assert sum(q.xdtype == "i8" for q in qs) > NQ // 3 and sum(q.xdtype == "f32" for q in qs) > NQ // 3


def test_graph_sample_vs_oracle(tm, uneven):
    qs, _, b = uneven
    out = tm.result_buffer(NQ)
    b.capture_graph(out)
    b.launch_graph()
    torch.cuda.synchronize()
    res = tm.decode_results(out)
    rng = np.random.default_rng(17)
    sample = rng.choice(NQ, 160, replace=False)
    exact_real = n_real = 0
    for i in sample:
        q = qs[int(i)]
        ref = O.match_query(q)
        if q.xdtype == "i8":
            check_int(b, int(i), q, res[int(i)], ref)
        else:
            n_real += 1
            exact_real += check_real(b, int(i), q, res[int(i)], ref)
    assert exact_real >= n_real - 2   # near-ties are rare


def test_alone_equals_in_batch(tm, uneven):
    qs, specs, b = uneven
    out = tm.result_buffer(NQ)
    b.run(out)
    torch.cuda.synchronize()
    res = tm.decode_results(out)
    for i in (0, 1, 2, 1000, NQ - 1):
        one = tm.Batch([specs[i]])
        o1 = tm.result_buffer(1)
        one.run(o1)
        torch.cuda.synchronize()
        r1 = tm.decode_results(o1)[0]
        # real signals too: their folds are cut into pieces fixed by the
        # signal alone, so the fp32 sums are the same in any batch
        assert r1 == res[i], (i, r1, res[i])
        if qs[i].xdtype != "i8":
            check_result(qs[i], r1, O.match_query(qs[i]))


def test_autotuned_batch_gives_the_same_results(tm, uneven):
    """The autotuner only changes the fold's stage ring: every result, real
    signals included, stays bit-identical (stage edges add +0.0 / +1 entries
    that count for nothing)."""
    qs, _, b = uneven
    plain = tm.result_buffer(NQ)
    b.run(plain)
    torch.cuda.synchronize()
    tiles = b.autotune(force=True)
    assert set(tiles) == {"i8", "f32"} and all(v in (16384, 32768, 65536) for v in tiles.values())
    out = tm.result_buffer(NQ)
    b.capture_graph(out)
    b.launch_graph()
    torch.cuda.synchronize()
    assert tm.decode_results(out) == tm.decode_results(plain)
    assert b.device_error() == 0


def test_pipelined_and_other_grids_equal_plain_run(tm, uneven):
    """tm_batch_set_grid + tm_batch_run_pipelined: every call's results
    (written one call later) equal the plain run's, bit for bit, for +-1
    and real signals alike (real folds follow fixed pieces, not shares)."""
    qs, specs, _ = uneven
    sub = specs[:512]
    b = tm.Batch(sub, pipelined=True)
    want = tm.result_buffer(len(sub))
    b.run(want)
    torch.cuda.synchronize()
    want = tm.decode_results(want)
    for F, C in ((0, 0), (120, 32), (97, 7), (152, 1)):
        b.set_grid(F, C)
        outs = [tm.result_buffer(len(sub)) for _ in range(3)]
        for k in range(5):
            b.run_pipelined(outs[k % 3])
        b.flush()
        torch.cuda.synchronize()
        for o in outs:
            assert tm.decode_results(o) == want, (F, C)
        plain = tm.result_buffer(len(sub))
        b.run(plain)
        torch.cuda.synchronize()
        assert tm.decode_results(plain) == want, (F, C)
    assert b.device_error() == 0
    b.close()


def test_full_range_sample_vs_oracle(tm):
    """Sixteen queries of the uneven mix over its whole length range (N up
    to 2^24, the range the 4096-query benchmark draws on the device), drawn
    on the host and checked against the oracle in one batch."""
    qs = W.uneven(seed=6100, n=16, logN=(20.0, 24.0))
    specs = [dict(x=torch.from_numpy(q.x).cuda(), t=torch.from_numpy(q.t).cuda(), N=q.N, K=q.K,
                  xdtype=q.xdtype, mode=q.mode) for q in qs]
    b = tm.Batch(specs, keep_corr=True)
    out = tm.result_buffer(len(qs))
    b.run(out)
    torch.cuda.synchronize()
    assert b.device_error() == 0
    res = tm.decode_results(out)
    assert max(q.N for q in qs) > (1 << 23)
    exact = n_real = 0
    for i, q in enumerate(qs):
        ref = O.match_query(q, corr="fft")
        if q.xdtype == "i8":
            check_int(b, i, q, res[i], ref)
        else:
            n_real += 1
            exact += check_real(b, i, q, res[i], ref)
    assert exact >= n_real - 1   # near-ties are rare
