"""The Thm. 2 sampling variant (TM_THM2_SAMPLING) on the GPU against the
oracle's ftm_thm2: folds of the zero-padded signal bit-exact (and their
periodic extension), circular correlations within 1e-5 normwise, maxima,
shift, status, |S1 ∩ S2| and score identical; the shared-memory and the
blocked correlation paths, M dividing N or not."""
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


CASES = [((1 << 20), 1024, "paper", True, "i8"), (300001, 500, "auto", False, "i8"),
         (65536, 1024, "paper", False, "i8"), ((1 << 22), 4096, "paper", False, "bits"),
         (200000, 20000, "paper", True, "i8"), (12345, 100, "auto", False, "bits")]


@pytest.mark.parametrize("N,K,mode,ambig,xdtype", CASES)
def test_thm2_vs_oracle(tm, N, K, mode, ambig, xdtype):
    qs = [W.planted_query(900 + s + N % 97, N, K, xdtype, flip_p=0.05, mode=mode, allow_ambig=ambig)
          for s in range(3)]
    for q in qs:
        q.meta["thm2"] = True
    specs = [dict(x=torch.from_numpy(q.x).cuda(), t=torch.from_numpy(q.t).cuda(), N=q.N, K=q.K, xdtype=xdtype,
                  mode=mode, allow_ambig=ambig, thm2=True) for q in qs]
    b = tm.Batch(specs, keep_corr=True)
    out = tm.result_buffer(len(qs))
    b.run(out)
    torch.cuda.synchronize()
    assert b.device_error() == 0
    res = tm.decode_results(out)
    for i, q in enumerate(qs):
        ref = O.match_query(q)
        P = b.infos[i]["P"]
        y = b.folds(i).cpu().numpy().astype(np.int64)
        r = b.corr(i).cpu().numpy().astype(np.float64)
        for j, (M, yr, rr) in enumerate(((ref["M1"], ref["y1"], ref["r1"]), (ref["M2"], ref["y2"], ref["r2"]))):
            ext = np.concatenate([yr, yr[:K - 1]])          # periodic extension
            assert np.array_equal(y[j * P: j * P + M + K - 1], ext), (i, j)
            got = r[j * P: j * P + M]
            assert np.abs(got - rr).max() <= 1e-5 * max(1.0, np.abs(rr).max())
        got = res[i]
        assert (got["m1"], got["m2"], got["shift"], got["status"] & 0xFF, got["n_cand"]) == \
            (ref["m1"], ref["m2"], ref["shift"], ref["status"], ref["n_cand"]), (i, got, ref)
        assert got["score"] == float(ref["score"])
