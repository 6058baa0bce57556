"""GPU path vs CPU oracle, element by element, through the C ABI.

Bar: folds (Eq. (2)) bit-exact in int32; FFT correlations r within 1e-5
normwise relative error of the fp64 oracle (max |dr| <= 1e-5 max |r|); the
step-7 maxima, the candidate count, the shift and its exact score identical.
"""
import numpy as np
import pytest
import torch

import oracle.ftm as O
import workloads as W

pytestmark = pytest.mark.gpu

R_TOL = 1e-5


@pytest.fixture(scope="module")
def tm():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1509_04863_gb300 import _build
    _build.build()
    import paper_1509_04863_gb300 as tm
    return tm


def _spec(q, dev="cuda"):
    return dict(x=torch.from_numpy(q.x).to(dev), t=torch.from_numpy(q.t).to(dev), N=q.N, K=q.K,
                xdtype=q.xdtype, mode=q.mode, M1=q.M1, M2=q.M2, allow_ambig=q.allow_ambig)


def run_batch(tm, queries, keep_corr=True):
    specs = [_spec(q) for q in queries]
    b = tm.Batch(specs, keep_corr=keep_corr)
    out = tm.result_buffer(len(queries))
    b.run(out)
    torch.cuda.synchronize()
    assert b.device_error() == 0
    return b, tm.decode_results(out), specs


def check(b, i, q, res, ref, check_r=True):
    P = b.infos[i]["P"]
    M1, M2, K = ref["M1"], ref["M2"], q.K
    y = b.folds(i).cpu().numpy()
    assert np.array_equal(y[:M1 + K - 1].astype(np.int64), ref["y1"]), f"query {i}: fold M1"
    assert np.array_equal(y[P:P + M2 + K - 1].astype(np.int64), ref["y2"]), f"query {i}: fold M2"
    if check_r:
        r = b.corr(i).cpu().numpy().astype(np.float64)
        for got, want in ((r[:M1], ref["r1"]), (r[P:P + M2], ref["r2"])):
            scale = max(1.0, float(np.abs(want).max()))
            err = float(np.abs(got - want).max())
            assert err <= R_TOL * scale, f"query {i}: r error {err} vs scale {scale}"
    assert res["m1"] == ref["m1"] and res["m2"] == ref["m2"], (i, res, ref["m1"], ref["m2"])
    assert res["r1"] == float(ref["r1"][ref["m1"]]) and res["r2"] == float(ref["r2"][ref["m2"]])
    assert res["n_cand"] == ref["n_cand"], (i, res["n_cand"], ref["n_cand"])
    assert (res["status"] & 0xFF) == ref["status"], (i, res["status"], ref["status"])
    assert res["shift"] == ref["shift"], (i, res["shift"], ref["shift"])
    assert res["score"] == float(ref["score"])


def test_single_query_workload(tm):
    """N = 65536 +-1 int8, K = 1024, noiseless, M1 = K, M2 = K+1."""
    qs = [W.single_query(seed) for seed in range(8)]
    b, res, _ = run_batch(tm, qs)
    hits = 0
    for i, q in enumerate(qs):
        ref = O.match_query(q)
        check(b, i, q, res[i], ref)
        hits += res[i]["shift"] == q.k_star
    assert hits >= 1


RAGGED = [
    # N, K, mode, allow_ambig, M1, M2
    (65536 + 7, 1024, "paper", False, 0, 0),      # ragged tail (< 16 bytes unfolded)
    (15, 3, "auto", False, 0, 0),                 # no 16-byte block at all
    (17, 16, "paper", False, 0, 0),               # M2 = N
    (4097, 4096, "paper", False, 0, 0),           # M1 = N - 1, one row
    (4096, 4096, "paper", False, 0, 0),           # M2 = N + 1
    (1000, 37, "paper", False, 0, 0),
    (123457, 2000, "paper", False, 0, 0),
    (20000, 5000, "paper", False, 0, 0),
    (100, 1, "auto", False, 0, 0),                # K = 1
    (1 << 20, 3000, "auto", False, 0, 0),
    (300000, 700, "auto", False, 0, 0),
    (99991, 300, "explicit", False, 331, 337),    # co-prime, not consecutive
    (1 << 22, 256, "paper", True, 0, 0),          # several CRT solutions
    (1 << 18, 8192, "paper", False, 0, 0),        # P = 16384, J = 2/3 units
    (50000, 8000, "auto", False, 0, 0),
    (300007, 100, "explicit", False, 20011, 20021),   # M + K - 1 > 16384 with one template block
    (1 << 20, 12000, "auto", False, 0, 0),            # FFT length 32768, blocked
    (200000, 20000, "paper", False, 0, 0),            # FFT length 65536: 3 template blocks
]


@pytest.mark.parametrize("N,K,mode,ambig,M1,M2", RAGGED)
def test_ragged_and_edge_sizes(tm, N, K, mode, ambig, M1, M2):
    qs = [W.planted_query(1000 + s + N % 97, N, K, "i8", flip_p=0.03, mode=mode, allow_ambig=ambig, M1=M1, M2=M2)
          for s in range(3)]
    b, res, _ = run_batch(tm, qs)
    for i, q in enumerate(qs):
        check(b, i, q, res[i], O.match_query(q))


def test_mixed_batch_and_composition_independence(tm):
    """Uneven shapes share fold CTAs; each result equals the one computed
    alone (the fold partition differs, the integer folds cannot)."""
    rng = np.random.default_rng(7)
    qs = []
    for s in range(40):
        N = int(2 ** rng.uniform(10, 20))
        K = int(min(N - 1, 2 ** rng.uniform(4, 11)))
        qs.append(W.planted_query(2000 + s, N, max(K, 1), "i8", flip_p=0.05, mode="auto"))
    b, res, _ = run_batch(tm, qs)
    for i, q in enumerate(qs):
        check(b, i, q, res[i], O.match_query(q))
    for i in (0, 13, 39):
        b1, r1, _ = run_batch(tm, [qs[i]])
        assert r1[0] == res[i]


def test_plan_match_api_and_host_path(tm):
    q = W.planted_query(5, 200003, 2048, "i8", flip_p=0.05)
    ref = O.match_query(q)
    s = _spec(q)
    p = tm.Plan(q.N, q.K, "i8", "paper")
    out = tm.result_buffer(1)
    p.match(s["x"], s["t"], out)
    torch.cuda.synchronize()
    r = tm.decode_results(out)[0]
    assert r["shift"] == ref["shift"] and r["m1"] == ref["m1"] and r["m2"] == ref["m2"]
    # a second call with other buffers re-binds the pointers
    q2 = W.planted_query(6, 200003, 2048, "i8", flip_p=0.05)
    s2 = _spec(q2)
    p.match(s2["x"], s2["t"], out)
    torch.cuda.synchronize()
    assert tm.decode_results(out)[0]["shift"] == O.match_query(q2)["shift"]
    # end to end from host buffers
    bh = tm.Batch([dict(x=None, t=None, N=q.N, K=q.K, xdtype="i8", mode="paper")], host_inputs=True)
    xh = torch.from_numpy(q.x).pin_memory()
    th = torch.from_numpy(q.t).pin_memory()
    oh = torch.zeros(tm.RESULT_BYTES // 8, dtype=torch.int64)
    bh.run_host([xh], [th], oh)
    rh = tm.decode_results(oh)[0]
    assert rh == r or (rh["shift"] == ref["shift"] and rh["m1"] == ref["m1"])


def test_repeat_runs_identical(tm):
    qs = W.batch64(seed=300, n=4, N=1 << 20, K=1024)
    b, res, specs = run_batch(tm, qs)
    out = tm.result_buffer(len(qs))
    for _ in range(3):
        b.run(out)
    torch.cuda.synchronize()
    assert tm.decode_results(out) == res


def test_batch64_full_size(tm):
    """64 queries, N = 2^24 +-1 int8, K = 4096, 5% template flips: every
    shift identical to the oracle; folds and r checked on a sample."""
    qs = W.batch64(seed=100, n=64)
    b, res, _ = run_batch(tm, qs)
    for i, q in enumerate(qs):
        ref = O.match_query(q)
        check(b, i, q, res[i], ref, check_r=(i % 16 == 0))


@pytest.mark.parametrize("K", [256, 1024, 4096, 8192, 16384])
def test_sweep_shapes(tm, K):
    """N = 2^22, flips p = 0.1, M1 = K, M2 = K+1 (several CRT solutions for
    K <= 1024; FFT length 2K = 32768 for K = 16384, correlated in blocks):
    shifts identical to the oracle."""
    qs = W.sweep(seed=1000 + K, K=K, n=6)
    b, res, _ = run_batch(tm, qs, keep_corr=False)
    for i, q in enumerate(qs):
        check(b, i, q, res[i], O.match_query(q), check_r=False)
