"""The multi-CTA path for long FFTs (one query on all SMs): FFT lengths from
2^15 (a query alone in its batch) up to 2^23 (K up to 2^22, beyond the
overlap-save correlation), against the oracle (FFT route in fp64, rounded
for integer data): folds bit-exact for +-1 signals, correlations within the
normwise tolerance, maxima, shift, status and score identical (reals: the
fp32 fold rules); the same queries through the one-CTA overlap-save path
(batches of more than eight) give identical results; degenerate signals
(every index tied) take the full rescoring; the Thm. 2 sampling; the
result carries no error flags."""
import numpy as np
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


def _spec(q, thm2=False):
    return dict(x=torch.from_numpy(q.x).cuda(), t=torch.from_numpy(q.t).cuda(), N=q.N, K=q.K, xdtype=q.xdtype,
                mode=q.mode, thm2=thm2)


def _run(tm, specs):
    b = tm.Batch(specs, keep_corr=True)
    out = tm.result_buffer(len(specs))
    b.run(out)
    torch.cuda.synchronize()
    assert b.device_error() == 0
    return b, tm.decode_results(out)


# (N, K, mode, dtype): FFT lengths 2^15 .. 2^23; 2^23 has two strided dims
CASES = [((1 << 17) + 3, 9000, "paper", "i8"), ((1 << 18) + 11, 20000, "auto", "i8"),
         (1 << 20, 1 << 18, "paper", "i8"), ((1 << 21) + 5, 300000, "paper", "f32"),
         (1 << 21, 1 << 19, "paper", "bits"), (1 << 22, 1 << 20, "paper", "f16"),
         (1 << 23, 1 << 21, "paper", "i8"), (1 << 24, 1 << 22, "paper", "i8")]


@pytest.mark.parametrize("N,K,mode,xdtype", CASES)
def test_large_vs_oracle(tm, N, K, mode, xdtype):
    ints = xdtype in ("i8", "bits")
    q = W.planted_query(2100 + N % 97 + K % 89, N, K, xdtype, flip_p=0.05 if ints else 0.0,
                        t_sigma=0.0 if ints else 0.3, mode=mode)
    b, res = _run(tm, [_spec(q)])
    assert b.infos[0]["P"] > 16384
    P = b.infos[0]["P"]
    nsd = 1 if P <= 1 << 22 else 2
    L = -(-N // b.infos[0]["M1"])
    fold_launches = 1 if (xdtype == "i8" and L <= 16) else 2   # int8 with few rows: no first stage
    assert b.stats()["launches_per_run"] == fold_launches + 1 + 2 * (nsd + 1) + nsd + 5
    ref = O.match_query(q, corr="fft")
    r = res[0]
    assert r["status"] & ~0xFF == 0, r
    if ints:
        check_int(b, 0, q, r, ref)
        assert r["shift"] == q.k_star
    else:
        check_real(b, 0, q, r, ref)


@pytest.mark.parametrize("N,K,xdtype", [((1 << 18) + 11, 20000, "i8"), ((1 << 19) + 1, 70000, "f32"),
                                        (1 << 20, 1 << 17, "bits")])
def test_large_equals_blocked(tm, N, K, xdtype):
    """One query alone (all-SM launches for one query) and the same query
    among nine (overlap-save blocks, one CTA per query, for 2^16 points; the
    all-SM launches over the whole batch for 2^18): the same folds and
    maxima; for +-1 signals every result field identical."""
    ints = xdtype != "f32"
    qs = [W.planted_query(2200 + s, N, K, xdtype, flip_p=0.05 if ints else 0.0, t_sigma=0.0 if ints else 0.3,
                          mode="paper") for s in range(9)]
    specs = [_spec(q) for q in qs]
    _, alone = _run(tm, specs[:1])
    _, many = _run(tm, specs)
    if ints:
        assert alone[0] == many[0]
    else:
        assert (alone[0]["m1"], alone[0]["m2"], alone[0]["shift"]) == (many[0]["m1"], many[0]["m2"], many[0]["shift"])
        assert abs(alone[0]["score"] - many[0]["score"]) <= 1e-9 * abs(many[0]["score"])


def test_large_degenerate_full_rescore(tm):
    """A constant signal and template: every correlation value ties, more
    than 4096 indices lie within the rounding bound, every index is rescored
    (TM_RF_FULL_RESCORE) and the smallest index wins, as in the oracle."""
    N, K = (1 << 17) + 3, 20000
    x = np.ones(N, dtype=np.int8)
    t = np.ones(K, dtype=np.float32)
    q = W.Query(x=x, xdtype="i8", N=N, K=K, t=t, k_star=0, mode="paper", M1=0, M2=0, allow_ambig=False, seed=0)
    b, res = _run(tm, [_spec(q)])
    ref = O.match_query(q, corr="fft")
    r = res[0]
    assert r["status"] & tm.TM_RF_FULL_RESCORE
    assert (r["m1"], r["m2"], r["shift"], r["n_cand"]) == (ref["m1"], ref["m2"], ref["shift"], ref["n_cand"])
    assert r["score"] == float(ref["score"])


@pytest.mark.parametrize("N,K", [((1 << 20) + 5, 1 << 17), ((1 << 19) + 77, 30000)])
def test_large_thm2(tm, N, K):
    q = W.planted_query(2300 + K % 7, N, K, "i8", flip_p=0.05, mode="paper")
    q.meta["thm2"] = True
    b, res = _run(tm, [_spec(q, thm2=True)])
    ref = O.match_query(q)
    r = res[0]
    P = b.infos[0]["P"]
    y = b.folds(0).cpu().numpy().astype(np.int64)
    for j, (M, key) in enumerate(((ref["M1"], "y1"), (ref["M2"], "y2"))):
        want = np.concatenate([ref[key], ref[key][:K - 1]])
        assert np.array_equal(y[j * P: j * P + M + K - 1], want)
    assert (r["m1"], r["m2"], r["shift"], r["status"] & 0xFF, r["n_cand"]) == \
        (ref["m1"], ref["m2"], ref["shift"], ref["status"], ref["n_cand"])
    assert r["score"] == float(ref["score"])


def test_large_graph_and_repeat(tm):
    """The long-FFT launches captured as a CUDA graph replay to the same
    results as plain runs, run after run, alone and in a batch of three."""
    qs = [W.planted_query(2400 + s, 1 << 20, 1 << 18, "i8", flip_p=0.05, mode="paper") for s in range(3)]
    for specs in ([_spec(qs[0])], [_spec(q) for q in qs]):
        b = tm.Batch(specs)
        plain = tm.result_buffer(len(specs))
        b.run(plain)
        torch.cuda.synchronize()
        want = tm.decode_results(plain)
        assert all(r["shift"] == q.k_star for r, q in zip(want, qs))
        for _ in range(2):
            b.run(plain)
            torch.cuda.synchronize()
            assert tm.decode_results(plain) == want
        out = tm.result_buffer(len(specs))
        b.capture_graph(out)
        for _ in range(3):
            out.zero_()
            b.launch_graph()
            torch.cuda.synchronize()
            assert tm.decode_results(out) == want
        assert b.device_error() == 0
