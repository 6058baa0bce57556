"""Slot sums ahead of the correlation (Eq. (2) across CTA shares).

A signal folded by many CTAs leaves one partial row per share (or per piece
of a real signal); a fold with at least 8 rows has them added into one row
by a many-CTA launch before the correlation. These tests check that such a
query (alone, so its fold spans every SM) gives the oracle's result, the
same result as inside a batch where its fold has few rows, and the same
result when the correlation is run twice on one fold (the sum goes to a row
of its own).
"""
import pytest
import torch

import oracle.ftm as O
import workloads as W
from parity import check_int, check_real

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tm():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1509_04863_gb300 import _build
    _build.build()
    import paper_1509_04863_gb300 as tm
    return tm


def _spec(q):
    return dict(x=torch.from_numpy(q.x).cuda(), t=torch.from_numpy(q.t).cuda(), N=q.N, K=q.K,
                xdtype=q.xdtype, mode=q.mode, M1=q.M1, M2=q.M2)


def _run(tm, qs):
    b = tm.Batch([_spec(q) for q in qs], keep_corr=True)
    out = tm.result_buffer(len(qs))
    b.run(out)
    torch.cuda.synchronize()
    assert b.device_error() == 0
    return b, tm.decode_results(out)


CASES = [
    # N, K, xdtype: one query's fold on every SM (int8 16 MiB: 152 rows;
    # bit-packed 2 MiB: 32 rows; fp32 16 MiB: 8 pieces of 2 MiB)
    (1 << 24, 4096, "i8"),
    (1 << 24, 4096, "bits"),
    (1 << 22, 2048, "f32"),
]


@pytest.mark.parametrize("N,K,xdtype", CASES, ids=[c[2] for c in CASES])
def test_many_rows_alone_vs_oracle_and_batch(tm, N, K, xdtype):
    ints = xdtype != "f32"
    q = W.planted_query(4100 + len(xdtype), N, K, xdtype, flip_p=0.05 if ints else 0.0,
                        t_sigma=0.0 if ints else 0.3, mode="paper")
    b1, r1 = _run(tm, [q])
    assert b1.stats()["launches_per_run"] == 3   # fold, slot sums, correlation
    ref = O.match_query(q)
    if ints:
        check_int(b1, 0, q, r1[0], ref)
    else:
        check_real(b1, 0, q, r1[0], ref)
    # among 40 other signals of its size a +-1 signal's fold has at most 5
    # rows (no slot sums); a real signal keeps its 8 pieces, summed alike
    others = [W.planted_query(4200 + s, N, K, xdtype, flip_p=0.05 if ints else 0.0,
                              t_sigma=0.0 if ints else 0.3, mode="paper") for s in range(40 if ints else 15)]
    bb, rb = _run(tm, others[:11] + [q] + others[11:])
    assert rb[11] == r1[0]
    y1 = b1.folds(0).cpu()
    yb = bb.folds(11).cpu()
    P = b1.infos[0]["P"]
    M1, M2 = b1.infos[0]["M1"], b1.infos[0]["M2"]
    assert torch.equal(y1[:M1 + K - 1], yb[:M1 + K - 1]) and torch.equal(y1[P:P + M2 + K - 1], yb[P:P + M2 + K - 1])


def test_correlate_twice_on_one_fold(tm):
    q = W.planted_query(4300, 1 << 23, 4096, "i8", flip_p=0.05, mode="paper")
    b = tm.Batch([_spec(q)])
    outs = [tm.result_buffer(1) for _ in range(3)]
    b.fold()
    b.correlate(outs[0])
    b.correlate(outs[1])
    b.run(outs[2])
    torch.cuda.synchronize()
    assert b.device_error() == 0
    res = [tm.decode_results(o)[0] for o in outs]
    assert res[0] == res[1] == res[2]
    assert res[0]["shift"] == O.match_query(q)["shift"]


def test_fine_pieces_real(tm):
    """TM_FINE_PIECES: a 16 MiB fp32 signal in 64 pieces of 256 KiB (8 of
    2 MiB without the flag): within the bars of the oracle, and the same
    alone and among other signals with the flag, bit for bit."""
    N, K = 1 << 22, 2048
    mk = lambda s: W.planted_query(s, N, K, "f32", t_sigma=0.3, mode="paper")
    q = mk(4400)
    spec = dict(_spec(q), fine_pieces=True)
    b1 = tm.Batch([spec], keep_corr=True)
    out = tm.result_buffer(1)
    b1.run(out)
    torch.cuda.synchronize()
    assert b1.device_error() == 0
    r1 = tm.decode_results(out)[0]
    check_real(b1, 0, q, r1, O.match_query(q))
    others = [dict(_spec(mk(4500 + s)), fine_pieces=True) for s in range(6)]
    bb = tm.Batch(others[:3] + [spec] + others[3:], keep_corr=True)
    outb = tm.result_buffer(len(others) + 1)
    bb.run(outb)
    torch.cuda.synchronize()
    assert bb.device_error() == 0
    assert tm.decode_results(outb)[3] == r1
    assert torch.equal(b1.folds(0).cpu(), bb.folds(3).cpu())
