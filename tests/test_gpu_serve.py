"""The continuous-batching server (tm_serve_*) on the GPU.

Requests on resident signals of every storage type go through the server
and come back equal to the CPU oracle's result for the same (signal,
template) pair (tests/parity.py: every field exact for +-1 signals; for real
signals r within 1e-5, the step-7 picks equal up to near-ties and steps 8-9
those of the oracle on the picks), and equal to the same queries run as
standalone batches; with the fold cache on, cached and uncached results both
meet the oracle bar; the same request alone and inside a mix gives the same
result;
an arena too small for the whole queue splits it into several iterations;
a request too large for the arena alone fails with TM_ENOMEM.
"""
import time

import numpy as np
import pytest
import torch

import oracle.ftm as O
import workloads as W
from parity import check_result

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tm():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1509_04863_gb300 import _build
    _build.build()
    import paper_1509_04863_gb300 as tm
    return tm


def _collect(srv, n, timeout_s=60.0):
    got = {}
    t0 = time.time()
    while len(got) < n and time.time() - t0 < timeout_s:
        for r in srv.poll(1024, timeout_us=20000):
            got[r["tag"]] = r
    assert len(got) == n, (len(got), n)
    return got


def _standalone(tm, q, x_dev):
    b = tm.Batch([dict(x=x_dev, t=torch.from_numpy(q.t).cuda(), N=q.N, K=q.K, xdtype=q.xdtype, mode=q.mode)])
    out = tm.result_buffer(1)
    b.run(out)
    torch.cuda.synchronize()
    return tm.decode_results(out)[0]


SIGNALS = [((1 << 20) + 3, "i8"), (1 << 20, "bits"), ((1 << 19) + 1, "f32"), ((1 << 18) + 5, "f16")]


@pytest.mark.parametrize("spin,fine", [(0, False), (200, False), (0, True)], ids=["sleep", "idle_spin", "fine_pieces"])
def test_server_matches_standalone(tm, spin, fine):
    srv = tm.Server(n_streams=2, max_batch=32, arena_bytes=1 << 30, idle_spin_us=spin, fine_pieces=fine)
    sigs, xs = [], []
    for k, (N, dt) in enumerate(SIGNALS):
        base = W.planted_query(9000 + k, N, 512, dt, mode="auto")
        # the device copy the standalone runs use
        xs.append(torch.from_numpy(base.x).cuda())
        sid = srv.register_signal(base.x, N, dt)   # host copy: the server keeps its own
        sigs.append((sid, base))
    reqs = {}
    rng = np.random.default_rng(3)
    tag = 0
    for rep in range(12):
        for k, (sid, base) in enumerate(sigs):
            # the registered signal, a new template window at a random shift
            K = int(rng.choice([256, 700, 1024, 2048]))
            k_star = int(rng.integers(0, base.N))
            t = W.flip_entries(rng, W.cyclic_window(_values(base), k_star, K), 0.03)
            q = W.Query(x=base.x, xdtype=base.xdtype, N=base.N, K=K, t=t, k_star=k_star, mode="auto")
            assert srv.submit(sid, q.t, tag=tag, mode="auto") == tm.TM_OK
            reqs[tag] = (k, q)
            tag += 1
    got = _collect(srv, len(reqs))
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["failed"] == 0 and st["iterations"] >= 2
    assert st["p50_us"] > 0 and st["p99_us"] >= st["p50_us"]
    exact = n_real = 0
    for t_, (k, q) in reqs.items():
        r = got[t_]
        assert r["req_status"] == tm.TM_OK and r["latency_us"] > 0
        exact_k = check_result(q, r, O.match_query(q))
        if q.xdtype in ("f16", "f32"):
            n_real += 1
            exact += exact_k
        ref = _standalone(tm, q, xs[k])
        if q.xdtype in ("i8", "bits"):
            assert {f: r[f] for f in ref} == ref, (t_, r, ref)
        else:
            check_result(q, ref, O.match_query(q))
    assert exact >= n_real - 2   # near-ties are rare
    srv.close()


def _values(q):
    import oracle.ftm as O
    return O.decode(q.x, q.xdtype, q.N).astype(np.float32)


def test_alone_and_in_the_mix(tm):
    srv = tm.Server(n_streams=2, max_batch=64, arena_bytes=1 << 30)
    qa = W.planted_query(77, (1 << 20) + 16, 1024, "i8", flip_p=0.05, mode="paper")
    sid = srv.register_signal(qa.x, qa.N, "i8")
    qb = W.planted_query(78, 1 << 19, 2048, "bits", flip_p=0.05, mode="auto")
    sid2 = srv.register_signal(qb.x, qb.N, "bits")
    qc = W.planted_query(79, (1 << 21) + 5, 1500, "f32", t_sigma=0.3, mode="auto")
    sid3 = srv.register_signal(qc.x, qc.N, "f32")
    srv.submit(sid, qa.t, tag=1, mode="paper")
    srv.submit(sid3, qc.t, tag=3, mode="auto")
    alone = _collect(srv, 2)
    for i in range(40):
        srv.submit(sid2, qb.t, tag=100 + i, mode="auto")
        if i == 20:
            srv.submit(sid, qa.t, tag=2, mode="paper")
            srv.submit(sid3, qc.t, tag=4, mode="auto")
    mixed = _collect(srv, 42)
    for ta, tb in ((1, 2), (3, 4)):
        a = {k: v for k, v in alone[ta].items() if k not in ("tag", "latency_us")}
        m = {k: v for k, v in mixed[tb].items() if k not in ("tag", "latency_us")}
        assert a == m, (ta, a, m)   # real signals too: their folds follow fixed pieces
    check_result(qc, mixed[4], O.match_query(qc))
    srv.close()


def test_arena_admission(tm):
    """A small arena runs the queue as several iterations; a request that
    alone exceeds it fails with TM_ENOMEM while the others complete."""
    srv = tm.Server(n_streams=1, max_batch=64, arena_bytes=4 << 20)
    q = W.planted_query(5, 1 << 20, 1024, "i8", flip_p=0.05, mode="paper")
    sid = srv.register_signal(q.x, q.N, "i8")
    big = W.planted_query(6, 1 << 22, 16384, "i8", mode="paper", allow_ambig=True)
    sid_big = srv.register_signal(big.x, big.N, "i8")
    for i in range(30):
        srv.submit(sid, q.t, tag=i, mode="paper")
    srv.submit(sid_big, big.t, tag=999, mode="paper", allow_ambig=True)
    got = _collect(srv, 31)
    assert got[999]["req_status"] == tm.TM_ENOMEM
    ok = [got[i] for i in range(30)]
    assert all(r["req_status"] == tm.TM_OK for r in ok)
    assert len({(r["shift"], r["m1"], r["m2"]) for r in ok}) == 1
    assert srv.stats()["iterations"] >= 2
    srv.close()


def test_submit_validation(tm):
    srv = tm.Server(n_streams=1, max_batch=8, arena_bytes=64 << 20)
    q = W.planted_query(1, 4096, 64, "i8")
    sid = srv.register_signal(q.x, q.N, "i8")
    with pytest.raises(tm.TMError) as e:
        srv.submit(sid + 7, q.t, tag=0)
    assert e.value.status == tm.TM_EINVAL
    with pytest.raises(tm.TMError) as e:
        srv.submit(sid, q.t[:16], tag=0, mode="paper")    # 16 * 17 <= 4096: needs allow_ambig
    assert e.value.status == tm.TM_EINVAL
    srv.close()


@pytest.mark.parametrize("fine", [False, True], ids=["pieces", "fine_pieces"])
def test_fold_cache(tm, fine):
    """Requests on resident signals whose moduli repeat are served from the
    fold cache (no O(N) fold): both servers meet the oracle bar and agree
    bit for bit (real folds follow fixed pieces), and the cache reports
    hits after the first fold of each (signal, M1, M2). With fine pieces
    the real signal's 4 MiB fold has 16 pieces, summed ahead by the slot-sum
    kernel."""
    # N = 2^20 + 3: automatic moduli M1 = max(K, 1024), so every K <= 1024
    # shares one pair
    N = (1 << 20) + 3
    base = [W.planted_query(4000 + k, N, 512, dt, mode="auto") for k, dt in enumerate(["i8", "f32", "bits"])]
    rng = np.random.default_rng(9)
    reqs = []
    for rnd in range(3):
        for k, q in enumerate(base):
            for K in (256, 700, 1000, 1024):
                k_star = int(rng.integers(0, N))
                t = W.flip_entries(rng, W.cyclic_window(_values(q), k_star, K), 0.03)
                reqs.append((k, K, t))
    outs = []
    for cache in (0, 64 << 20):
        srv = tm.Server(n_streams=2, max_batch=8, arena_bytes=1 << 28, fold_cache_bytes=cache, fine_pieces=fine)
        ids = [srv.register_signal(q.x, q.N, q.xdtype) for q in base]
        got = {}
        for i, (k, K, t) in enumerate(reqs):
            assert srv.submit(ids[k], t, tag=i, mode="auto") == tm.TM_OK
            if i % 12 == 11:   # let earlier rounds finish so later ones can hit
                got.update(_collect(srv, i + 1 - len(got)))
        got.update(_collect(srv, len(reqs) - len(got)))
        st = srv.stats()
        outs.append((got, st))
        srv.close()
    (plain, st0), (cached, st1) = outs
    assert st0["fold_cache_hits"] == 0
    assert st1["fold_cache_hits"] >= len(reqs) // 2 and st1["failed"] == 0
    fields = ("shift", "status", "m1", "m2", "r1", "r2", "score", "n_cand")
    for i, (k, K, t) in enumerate(reqs):
        a, b = plain[i], cached[i]
        assert a["req_status"] == b["req_status"] == tm.TM_OK
        q = W.Query(x=base[k].x, xdtype=base[k].xdtype, N=N, K=K, t=t, k_star=0, mode="auto")
        ref = O.match_query(q)
        check_result(q, a, ref)
        check_result(q, b, ref)
        # real folds follow fixed pieces: cached and uncached alike, bit for bit
        assert {f: a[f] for f in fields} == {f: b[f] for f in fields}, (i, a, b)


def test_long_fft_requests(tm):
    """Requests whose FFT exceeds the overlap-save range (P = 2^19, the
    all-SM path) and others in the overlap-save range go through the server
    among ordinary ones and equal the standalone runs (+-1 signals)."""
    srv = tm.Server(n_streams=2, max_batch=16, arena_bytes=1 << 30)
    long_q = W.planted_query(31, 1 << 20, 1 << 18, "i8", flip_p=0.05, mode="paper")
    mid_q = W.planted_query(32, 1 << 21, 40000, "i8", flip_p=0.05, mode="paper")
    small_q = W.planted_query(33, 1 << 20, 1024, "i8", flip_p=0.05, mode="paper")
    xs, sids = [], []
    for q in (long_q, mid_q, small_q):
        xs.append(torch.from_numpy(q.x).cuda())
        sids.append(srv.register_signal(q.x, q.N, "i8"))
    order = [0, 2, 1, 2, 0, 1, 2, 2]
    for tag, k in enumerate(order):
        assert srv.submit(sids[k], (long_q, mid_q, small_q)[k].t, tag=tag, mode="paper") == tm.TM_OK
    got = _collect(srv, len(order))
    for tag, k in enumerate(order):
        q = (long_q, mid_q, small_q)[k]
        r = got[tag]
        assert r["req_status"] == tm.TM_OK
        ref = _standalone(tm, q, xs[k])
        assert {f: r[f] for f in ref} == ref, (tag, r, ref)
        if k < 2:   # K^2 / ln K well above N: the planted shift comes back
            assert r["shift"] == q.k_star
    srv.close()


def test_submit_many(tm):
    """tm_serve_submit_many queues a burst in one call; every result equals
    the oracle's, and an unknown signal id stops the burst after the valid
    prefix."""
    srv = tm.Server(n_streams=2, max_batch=64, arena_bytes=1 << 28)
    base = [W.planted_query(8100 + k, (1 << 19) + 11 * k, 512, dt, mode="auto")
            for k, dt in enumerate(["i8", "f32", "bits"])]
    ids = [srv.register_signal(q.x, q.N, q.xdtype) for q in base]
    rng = np.random.default_rng(21)
    qs, sig, ts = [], [], []
    for i in range(30):
        k = i % 3
        K = int(rng.choice([300, 512, 700]))
        t = W.flip_entries(rng, W.cyclic_window(_values(base[k]), int(rng.integers(0, base[k].N)), K), 0.03)
        qs.append(W.Query(x=base[k].x, xdtype=base[k].xdtype, N=base[k].N, K=K, t=t, k_star=0, mode="auto"))
        sig.append(ids[k])
        ts.append(np.ascontiguousarray(t, dtype=np.float32))
    assert srv.submit_many(sig, ts, list(range(30)), mode="auto") == 30
    got = _collect(srv, 30)
    for i, q in enumerate(qs):
        assert got[i]["req_status"] == tm.TM_OK
        check_result(q, got[i], O.match_query(q))
    got_all = dict(got)
    assert srv.submit_many([ids[0], 99, ids[1]], ts[:3], [100, 101, 102], mode="auto") == 1
    got = _collect(srv, 1)
    assert got[100]["req_status"] == tm.TM_OK
    with pytest.raises(tm.TMError):
        srv.submit_many([99], ts[:1], [200], mode="auto")
    # the array forms: the same 30 requests again, results as a structured array
    n = len(ts)
    assert srv.submit_many_arrays(np.array(sig, dtype=np.int32), np.array([t.ctypes.data for t in ts], dtype=np.uint64),
                                  np.array([t.shape[0] for t in ts], dtype=np.int32),
                                  np.arange(1000, 1000 + n, dtype=np.uint64), mode="auto") == n
    rows, t0 = [], time.time()
    while sum(len(r) for r in rows) < n and time.time() - t0 < 60:
        rows.append(srv.poll_array(64, timeout_us=20000))
    arr = np.concatenate(rows)
    assert len(arr) == n and np.all(arr["status"] == tm.TM_OK)
    for row in arr:
        i = int(row["tag"]) - 1000
        assert int(row["r"]["shift"]) == got_all[i]["shift"] and int(row["r"]["m1"]) == got_all[i]["m1"]
    srv.close()
