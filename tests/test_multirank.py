"""The multi-GPU host path on CPU: two gloo ranks shard a batch of queries,
each runs its share (here through the CPU oracle, as the data path needs no
collective), and the gathered results equal the single-process ones; the job
time is the maximum over ranks."""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_1509_04863_gb300.parallel import shard_range


def test_shard_range_covers_exactly_once():
    for n in (0, 1, 7, 64, 4097):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                s, e = shard_range(n, world, r)
                assert 0 <= s <= e <= n
                seen.extend(range(s, e))
            assert seen == list(range(n))
            sizes = [shard_range(n, world, r)[1] - shard_range(n, world, r)[0] for r in range(world)]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import json

    import torch.distributed as dist

    import oracle.ftm as O
    import workloads as W
    from paper_1509_04863_gb300.parallel import gather_results, max_over_ranks, rank_env, shard_range

    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = rank_env()
    assert (r, w) == (rank, world)
    qs = W.batch64(seed=40, n=7, N=1 << 14, K=128, flip_p=0.02)
    s, e = shard_range(len(qs), w, r)
    mine = [O.match_query(qs[i])["shift"] for i in range(s, e)]
    allres = gather_results(mine, len(qs))
    slowest = max_over_ranks(float(10 + rank))
    dist.barrier()
    if rank == 0:
        with open(out_path, "w") as f:
            json.dump({"results": allres, "slowest": slowest}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process(tmp_path):
    import json

    import oracle.ftm as O
    import workloads as W

    out = str(tmp_path / "res.json")
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    got = json.load(open(out))
    want = [O.match_query(q)["shift"] for q in W.batch64(seed=40, n=7, N=1 << 14, K=128, flip_p=0.02)]
    assert got["results"] == want
    assert got["slowest"] == 11.0


# ---------------------------------------------------------------- one signal in slices
class OracleSliceOps:
    """match_sliced's four steps from the oracle (CPU), for the gloo test."""

    def __init__(self, N, M1, M2, t):
        import oracle.ftm as O
        self.O, self.N, self.M, self.t = O, N, (M1, M2), O.template_values(t)
        self.K = self.t.shape[0]

    def fold_slice(self, xs, n0, length):
        import torch
        ys = [self.O.fold_slice(xs, n0, self.N, M, self.K) for M in self.M]
        return torch.from_numpy(np.concatenate(ys).astype(np.int64))

    def correlate_folds(self, y):
        O, (M1, M2), K = self.O, self.M, self.K
        y = y.numpy()
        y1, y2 = y[:M1 + K - 1], y[M1 + K - 1:]
        m1 = O.argmax_first(O.correlate(y1, self.t, M1))
        m2 = O.argmax_first(O.correlate(y2, self.t, M2))
        return {"m1": m1, "m2": m2, "status": 0x400}

    def candidates(self, res):
        O, (M1, M2) = self.O, self.M
        return sorted(O.candidate_set(res["m1"], M1, self.N) & O.candidate_set(res["m2"], M2, self.N))

    def score_slice(self, xs, n0, length, m):
        import torch
        return torch.tensor([float(self.O.tx_slice(xs, n0, self.N, self.t, int(v))) for v in m.tolist()],
                            dtype=torch.float64)


SLICE_CASES = [dict(seed=31, N=20003, K=200, mode="paper", ambig=False),
               dict(seed=32, N=5000, K=40, mode="paper", ambig=True)]


def _slice_rank_main(rank, world, port, out_path):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import json

    import torch.distributed as dist

    import oracle.ftm as O
    import workloads as W
    from paper_1509_04863_gb300.parallel import match_sliced, slice_bounds

    dist.init_process_group("gloo", rank=rank, world_size=world)
    got = []
    for c in SLICE_CASES:
        q = W.planted_query(c["seed"], c["N"], c["K"], "i8", flip_p=0.05, mode=c["mode"], allow_ambig=c["ambig"])
        M1, M2 = O.plan(q.N, q.K, q.mode, allow_ambig=q.allow_ambig)
        x = O.decode(q.x, q.xdtype, q.N)
        n0, n1 = slice_bounds(q.N, world, rank)
        res = match_sliced(OracleSliceOps(q.N, M1, M2, q.t), x[n0:n1], n0, n1 - n0)
        if rank == 0:
            got.append({k: res[k] for k in ("m1", "m2", "shift", "status", "score")})
    dist.barrier()
    if rank == 0:
        with open(out_path, "w") as f:
            json.dump(got, f)
    dist.destroy_process_group()


def test_sliced_signal_two_gloo_ranks(tmp_path):
    import json

    import oracle.ftm as O
    import workloads as W

    out = str(tmp_path / "sliced.json")
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_slice_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    got = json.load(open(out))
    for c, g in zip(SLICE_CASES, got):
        q = W.planted_query(c["seed"], c["N"], c["K"], "i8", flip_p=0.05, mode=c["mode"], allow_ambig=c["ambig"])
        ref = O.match_query(q)
        assert (g["m1"], g["m2"], g["shift"], g["status"]) == (ref["m1"], ref["m2"], ref["shift"], ref["status"])
        assert g["score"] == float(ref["score"])
    assert got[1]["status"] == O.RESOLVED or got[0]["status"] == O.FOUND


def test_slice_bounds_partition():
    from paper_1509_04863_gb300.parallel import slice_bounds
    for N in (1, 15, 16, 17, 20003, 1 << 20):
        for world in (1, 2, 3, 8):
            b = [slice_bounds(N, world, r) for r in range(world)]
            assert b[0][0] == 0 and b[-1][1] == N
            for (a0, a1), (c0, c1) in zip(b[:-1], b[1:]):
                assert a1 == c0
            assert all(n0 % 16 == 0 or n0 == N for n0, _ in b)
