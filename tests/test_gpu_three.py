"""Three co-prime moduli (TM_THREE_MODULI, Thm. 4) on the GPU against the
oracle's ftm_multi: the three folds bit-exact for +-1 signals, the FFT
correlations within 1e-5 normwise, the three maxima, |S1 ∩ S2 ∩ S3|, shift,
status and score identical; a planted strong window in a real signal is
recovered uniquely where two moduli leave several members; a mixed batch
of two- and three-moduli queries equals the queries run alone."""
import numpy as np
import pytest
import torch

import oracle.ftm as O
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tm():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1509_04863_gb300 import _build
    _build.build()
    import paper_1509_04863_gb300 as tm
    return tm


def _spec(q, three=True):
    return dict(x=torch.from_numpy(q.x).cuda(), t=torch.from_numpy(q.t).cuda(), N=q.N, K=q.K, xdtype=q.xdtype,
                mode=q.mode, allow_ambig=q.allow_ambig, three=three)


CASES = [(1 << 20, 128, "paper", False, "i8"), (300001, 500, "auto", False, "i8"),
         ((1 << 22) + 5, 1024, "paper", False, "bits"), (65536 + 7, 32, "paper", True, "i8"),
         (1 << 18, 4095, "paper", False, "i8")]


@pytest.mark.parametrize("N,K,mode,ambig,xdtype", CASES)
def test_three_moduli_vs_oracle(tm, N, K, mode, ambig, xdtype):
    qs = [W.planted_query(1200 + s + N % 89, N, K, xdtype, flip_p=0.03, mode=mode, allow_ambig=ambig)
          for s in range(3)]
    for q in qs:
        q.meta["three"] = True
    b = tm.Batch([_spec(q) for q in qs], keep_corr=True)
    out = tm.result_buffer(len(qs))
    b.run(out)
    torch.cuda.synchronize()
    assert b.device_error() == 0
    res = tm.decode_results(out)
    for i, q in enumerate(qs):
        ref = O.match_query(q)
        P = b.infos[i]["P"]
        Ms = ref["moduli"]
        assert (b.infos[i]["M1"], b.infos[i]["M2"], b.infos[i]["M3"]) == Ms
        y = b.folds(i).cpu().numpy().astype(np.int64)
        r = b.corr(i).cpu().numpy().astype(np.float64)
        for j, M in enumerate(Ms):
            assert np.array_equal(y[j * P: j * P + M + K - 1], ref["ys"][j]), (i, j)
            rr = ref["rs"][j].astype(np.float64)
            assert np.abs(r[j * P: j * P + M] - rr).max() <= 1e-5 * max(1.0, np.abs(rr).max())
        got = res[i]
        assert (got["m1"], got["m2"], got["m3"]) == tuple(ref["ms"]), (i, got, ref["ms"])
        assert (got["shift"], got["status"] & 0xFF, got["n_cand"]) == (ref["shift"], ref["status"], ref["n_cand"])
        assert got["score"] == float(ref["score"])
        assert (got["r1"], got["r2"], got["r3"]) == tuple(float(ref["rs"][j][ref["ms"][j]]) for j in range(3))


def test_three_moduli_recover_a_strong_window(tm):
    rng = np.random.default_rng(8)
    N, K = 300000, 257
    x = (0.01 * rng.standard_normal(N)).astype(np.float32)
    k_star = 123457
    t = np.where(rng.random(K) < 0.5, 1.0, -1.0).astype(np.float32)
    x[(np.arange(K) + k_star) % N] = t
    q = W.Query(x=x, xdtype="f32", N=N, K=K, t=t, k_star=k_star, mode="paper", allow_ambig=True)
    two = tm.Batch([_spec(q, three=False)])
    three = tm.Batch([_spec(q, three=True)])
    o2, o3 = tm.result_buffer(1), tm.result_buffer(1)
    two.run(o2)
    three.run(o3)
    torch.cuda.synchronize()
    r2, r3 = tm.decode_results(o2)[0], tm.decode_results(o3)[0]
    assert r2["n_cand"] > 1 and r2["shift"] == k_star and r2["status"] & 0xFF == tm.TM_RESOLVED
    assert r3["n_cand"] == 1 and r3["shift"] == k_star and r3["status"] & 0xFF == tm.TM_FOUND


def test_mixed_two_and_three_moduli_batch(tm):
    qs = [W.planted_query(1300 + s, (1 << 19) + 3 * s, 256 + 64 * s, "i8", flip_p=0.03, mode="auto")
          for s in range(6)]
    specs = [_spec(q, three=(s % 2 == 1)) for s, q in enumerate(qs)]
    b = tm.Batch(specs)
    out = tm.result_buffer(len(qs))
    b.run(out)
    torch.cuda.synchronize()
    res = tm.decode_results(out)
    for s, sp in enumerate(specs):
        one = tm.Batch([sp])
        o1 = tm.result_buffer(1)
        one.run(o1)
        torch.cuda.synchronize()
        assert tm.decode_results(o1)[0] == res[s]
