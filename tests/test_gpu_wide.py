"""Moduli too wide for the streaming fold's register-resident columns
(K >= 2^14, up to FFT lengths of 2^17 here): the entry-by-entry fold and the
overlap-save correlation against the oracle (FFT route in fp64, rounded for
integer data): folds bit-exact for +-1 signals and within 1e-5 for reals,
maxima, shift, status, score identical; also with the Thm. 2 sampling.
The batches hold more than eight such queries (each pair five times), so
FFTs of 2^15 and 2^16 points take the one-CTA-per-query overlap-save
path; 2^17 points and more, and smaller batches, take the all-SM launches
(test_gpu_large.py)."""
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


CASES = [(1 << 21, 32768, "paper", "i8", False), ((1 << 20) + 3, 40000, "auto", "i8", False),
         (1 << 22, 20000, "paper", "f32", False), (1 << 21, 17000, "paper", "bits", False),
         ((1 << 21) + 5, 30000, "paper", "i8", True)]


@pytest.mark.parametrize("N,K,mode,xdtype,thm2", CASES)
def test_wide_moduli_vs_oracle(tm, N, K, mode, xdtype, thm2):
    ints = xdtype in ("i8", "bits")
    qs = [W.planted_query(1500 + s + N % 83, N, K, xdtype, flip_p=0.05 if ints else 0.0,
                          t_sigma=0.0 if ints else 0.3, mode=mode) for s in range(2)]
    specs = []
    for q in qs:
        q.meta["thm2"] = thm2
        specs.append(dict(x=torch.from_numpy(q.x).cuda(), t=torch.from_numpy(q.t).cuda(), N=q.N, K=q.K,
                          xdtype=xdtype, mode=mode, thm2=thm2))
    b = tm.Batch(specs * 5, keep_corr=True)
    if b.infos[0]["P"] < 1 << 17:   # ten queries of 2^15 or 2^16 points: overlap-save, one CTA per query
        assert b.stats()["launches_per_run"] in (2, 3)   # entry-by-entry fold (one or two) + overlap-save
    out = tm.result_buffer(5 * len(qs))
    b.run(out)
    torch.cuda.synchronize()
    assert b.device_error() == 0
    res = tm.decode_results(out)
    for i in range(len(qs), 5 * len(qs)):
        assert res[i] == res[i % len(qs)]
    for i, q in enumerate(qs):
        ref = O.match_query(q, corr="fft") if not thm2 else O.match_query(q)
        P = b.infos[i]["P"]
        y = b.folds(i).cpu().numpy().astype(np.float64)
        for j, (M, key) in enumerate(((ref["M1"], "y1"), (ref["M2"], "y2"))):
            want = ref[key].astype(np.float64)
            if thm2:
                want = np.concatenate([want, want[:K - 1]])
            got = y[j * P: j * P + M + K - 1]
            if ints:
                assert np.array_equal(got, want), (i, j)
            else:
                assert np.abs(got - want).max() <= 1e-5 * max(1.0, np.abs(want).max())
        got = res[i]
        if ints:
            assert (got["m1"], got["m2"], got["shift"], got["status"] & 0xFF, got["n_cand"]) == \
                (ref["m1"], ref["m2"], ref["shift"], ref["status"], ref["n_cand"]), (i, got)
            assert got["score"] == float(ref["score"])
        else:
            assert got["shift"] == ref["shift"] or abs(got["r1"] - float(ref["r1"][ref["m1"]])) <= 1e-3 * abs(got["r1"])
