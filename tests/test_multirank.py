"""The multi-GPU host path on CPU: two gloo ranks shard a batch of queries,
each runs its share (here through the CPU oracle, as the data path needs no
collective), and the gathered results equal the single-process ones; the job
time is the maximum over ranks."""
import os
import socket

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
