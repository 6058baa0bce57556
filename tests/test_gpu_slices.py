"""One signal cut into slices (the multi-GPU split of one long signal), on one
GPU: the library's slice folds equal the oracle's restricted folds and add
up to the whole signal's folds (bit-exact for +-1 signals); steps 4-8 on
the summed folds give the oracle's maxima; the slices' partial scores add
up to the exact scores; the whole protocol (match_sliced with the library's
operations) equals tm_match."""
import numpy as np
import pytest
import torch

import oracle.ftm as O
import workloads as W

pytestmark = pytest.mark.gpu

BITS = {"i8": 8, "bits": 1, "f16": 16, "f32": 32}


@pytest.fixture(scope="module")
def tm():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1509_04863_gb300 import _build
    _build.build()
    import paper_1509_04863_gb300 as tm
    return tm


def _cuts(N, xdtype, n, seed):
    """n slices with starts on 16-byte boundaries of the signal."""
    a = 128 // BITS[xdtype]
    rng = np.random.default_rng(seed)
    inner = sorted({int(v) // a * a for v in rng.integers(a, max(a + 1, N - 1), n - 1)} - {0})
    b = [0, *[v for v in inner if v < N], N]
    return list(zip(b[:-1], b[1:]))


def _storage(x_dev, xdtype, a, b):
    if xdtype == "bits":
        return x_dev[a // 8: (b + 7) // 8]
    return x_dev[a:b]


@pytest.mark.parametrize("xdtype,N,K,nsl", [("i8", (1 << 20) + 5, 1024, 3), ("i8", 300001, 700, 5),
                                            ("bits", (1 << 19) + 77, 512, 3), ("f32", 200003, 900, 4),
                                            ("f16", 100000, 333, 2)])
def test_slice_folds_add_up(tm, xdtype, N, K, nsl):
    ints = xdtype in ("i8", "bits")
    q = W.planted_query(40 + nsl, N, K, xdtype, flip_p=0.05 if ints else 0.0, t_sigma=0.0 if ints else 0.3,
                        mode="auto")
    plan = tm.Plan(N, K, xdtype, "auto")
    info = plan.info
    P, M1, M2 = info["P"], info["M1"], info["M2"]
    x = O.decode(q.x, xdtype, N)
    x_dev = torch.from_numpy(q.x).cuda()
    t_dev = torch.from_numpy(q.t).cuda()
    ydt = torch.int32 if ints else torch.float32
    ysum = torch.zeros(2 * P, dtype=ydt, device="cuda")
    cuts = _cuts(N, xdtype, nsl, N)
    for a, b in cuts:
        y = torch.full((2 * P,), 7, dtype=ydt, device="cuda")   # every entry gets written
        plan.fold_slice(_storage(x_dev, xdtype, a, b), a, b - a, y)
        torch.cuda.synchronize()
        yh = y.cpu().numpy().astype(np.float64)
        for j, M in ((0, M1), (1, M2)):
            want = O.fold_slice(x[a:b], a, N, M, K).astype(np.float64)
            got = yh[j * P: j * P + M + K - 1]
            if ints:
                assert np.array_equal(got, want), (a, b, j)
            else:
                assert np.abs(got - want).max() <= 1e-5 * max(1.0, np.abs(want).max())
            assert not yh[j * P + M + K - 1: (j + 1) * P].any()
        ysum += y
    yh = ysum.cpu().numpy().astype(np.float64)
    for j, M in ((0, M1), (1, M2)):
        want = O.fold(x, M, K).astype(np.float64)
        got = yh[j * P: j * P + M + K - 1]
        if ints:
            assert np.array_equal(got, want)
        else:
            assert np.abs(got - want).max() <= 1e-5 * max(1.0, np.abs(want).max())

    # steps 4-8 on the summed folds, then the partial scores of step 9
    ref = O.match_query(q)
    out = tm.result_buffer(1)
    plan.correlate_folds(ysum, t_dev, out)
    torch.cuda.synchronize()
    res = tm.decode_results(out)[0]
    if ints:
        assert (res["m1"], res["m2"], res["n_cand"]) == (ref["m1"], ref["m2"], ref["n_cand"])
    members = tm.tm_crt_candidates(N, M1, M2, res["m1"], res["m2"])
    assert len(members) == res["n_cand"]
    if members:
        assert res["status"] & tm.TM_RF_SCORE_PENDING
        m = torch.tensor(members, dtype=torch.int64, device="cuda")
        tot = torch.zeros(len(members), dtype=torch.float64, device="cuda")
        for a, b in cuts:
            sc = torch.zeros(len(members), dtype=torch.float64, device="cuda")
            plan.score_slice(_storage(x_dev, xdtype, a, b), a, b - a, t_dev, m, sc)
            tot += sc
        tot = tot.cpu().numpy()
        want = np.array([float(O.tx_at(x, O.template_values(q.t), v)) for v in members])
        assert np.allclose(tot, want, rtol=1e-12, atol=1e-9), (tot, want)
        if ints:
            assert np.array_equal(tot, want)


@pytest.mark.parametrize("xdtype", ["i8", "f32"])
def test_match_sliced_single_process_equals_match(tm, xdtype):
    """match_sliced without a process group (one slice) = tm_match."""
    from paper_1509_04863_gb300.parallel import LibSliceOps, match_sliced
    N, K = (1 << 18) + 3, 600
    q = W.planted_query(77, N, K, xdtype, flip_p=0.05 if xdtype == "i8" else 0.0,
                        t_sigma=0.3 if xdtype == "f32" else 0.0, mode="auto")
    plan = tm.Plan(N, K, xdtype, "auto")
    x_dev = torch.from_numpy(q.x).cuda()
    t_dev = torch.from_numpy(q.t).cuda()
    out = tm.result_buffer(1)
    plan.match(x_dev, t_dev, out)
    torch.cuda.synchronize()
    want = tm.decode_results(out)[0]
    got = match_sliced(LibSliceOps(plan, t_dev), x_dev, 0, N)
    assert (got["shift"], got["status"], got["m1"], got["m2"]) == \
        (want["shift"], want["status"], want["m1"], want["m2"])
    assert abs(got["score"] - want["score"]) <= 1e-9 * max(1.0, abs(want["score"]))
