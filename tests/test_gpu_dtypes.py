"""GPU path vs CPU oracle for every signal storage type, through the C ABI.

- bit-packed +-1: folds, correlations' argmax, shifts bit-exact (integers);
- fp32 and fp16 storage (real signals, real templates): folds and FFT
  correlations within 1e-5 normwise of the fp64 oracle (the oracle decodes
  the stored values exactly, so storage rounding is common to both sides);
  the step-7 maxima and the shift identical unless the oracle's top two
  correlations lie within the fp32 error of the fold, in which case the GPU
  pick must be one of those near-maximal entries;
- a mixed batch (all four types, uneven N and K, automatic moduli) equals
  the per-query results bit for bit, real signals included.
"""
import numpy as np
import pytest
import torch

import oracle.ftm as O
import workloads as W

pytestmark = pytest.mark.gpu

from parity import check_int, check_real, TOL  # noqa: F401


@pytest.fixture(scope="module")
def tm():
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1509_04863_gb300 import _build
    _build.build()
    import paper_1509_04863_gb300 as tm
    return tm


def _spec(q):
    return dict(x=torch.from_numpy(q.x).cuda(), t=torch.from_numpy(q.t).cuda(), N=q.N, K=q.K, xdtype=q.xdtype,
                mode=q.mode, M1=q.M1, M2=q.M2, allow_ambig=q.allow_ambig)


def _run(tm, qs):
    b = tm.Batch([_spec(q) for q in qs], keep_corr=True)
    out = tm.result_buffer(len(qs))
    b.run(out)
    torch.cuda.synchronize()
    assert b.device_error() == 0
    return b, tm.decode_results(out)


@pytest.mark.parametrize("N,K", [(1 << 20, 2048), ((1 << 18) + 77, 1024), (5000, 300), (100, 20), (1 << 22, 4096)])
def test_bitpacked_exact(tm, N, K):
    qs = [W.planted_query(300 + s + N % 101, N, K, "bits", flip_p=0.05, mode="auto") for s in range(3)]
    b, res = _run(tm, qs)
    for i, q in enumerate(qs):
        check_int(b, i, q, res[i], O.match_query(q))


def test_bitpacked_batch64_shape(tm):
    """The bit-packed variant of the 64-query workload (N = 2^24, K = 4096)
    on a sample of 8 queries."""
    qs = W.batch64(seed=100, n=8, xdtype="bits")
    b, res = _run(tm, qs)
    for i, q in enumerate(qs):
        check_int(b, i, q, res[i], O.match_query(q))


@pytest.mark.parametrize("xdtype", ["f32", "f16"])
@pytest.mark.parametrize("N,K", [(1 << 20, 2048), ((1 << 18) + 5, 512), (3000, 200), (1 << 22, 8000),
                                 ((1 << 20) + 3, 12000)])
def test_real_signals(tm, xdtype, N, K):
    qs = [W.planted_query(500 + s + N % 89, N, K, xdtype, t_sigma=0.3, mode="auto") for s in range(3)]
    b, res = _run(tm, qs)
    exact = 0
    for i, q in enumerate(qs):
        exact += check_real(b, i, q, res[i], O.match_query(q))
    assert exact >= 2   # near-ties are rare


def test_mixed_types_uneven_batch(tm):
    """Uneven batch with all four storage types: results equal per-query runs."""
    rng = np.random.default_rng(11)
    qs = []
    for s in range(24):
        N = int(2 ** rng.uniform(12, 20))
        K = int(min(N - 1, 2 ** rng.uniform(6, 11)))
        dt = ("i8", "bits", "f16", "f32")[s % 4]
        qs.append(W.planted_query(700 + s, N, K, dt, flip_p=0.05 if dt in ("i8", "bits") else 0.0,
                                  t_sigma=0.3 if dt in ("f16", "f32") else 0.0, mode="auto"))
    b, res = _run(tm, qs)
    assert b.stats()["launches_per_run"] in (5, 6)   # 4 fold groups, correlation (+ slot sums of folds with >= 8 rows)
    for i, q in enumerate(qs):
        ref = O.match_query(q)
        if q.xdtype in ("i8", "bits"):
            check_int(b, i, q, res[i], ref)
        else:
            check_real(b, i, q, res[i], ref)
    for i in (1, 2, 3, 4):
        # alone and in the batch, bit for bit (real folds follow fixed pieces)
        b1, r1 = _run(tm, [qs[i]])
        assert r1[0] == res[i], (i, r1[0], res[i])
