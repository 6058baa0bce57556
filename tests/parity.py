"""Parity rules shared by the GPU tests: a GPU result against the CPU
oracle's on the same seeded inputs.

+-1 signals (int8, bit-packed): folds bit-exact, FFT correlations within
1e-5 normwise, step-7 maxima, |S1 ∩ S2| and shift identical; the exact r
values and score identical for integral templates (integers), within fp64
rounding of their K-term sums for real templates.

Real signals (fp32 or fp16 storage; the oracle decodes the stored values
exactly, so storage rounding is common to both sides): folds and FFT
correlations within 1e-5 normwise of the fp64 oracle. The GPU's step 7 is
exact for its own fp32 folds; against the fp64 folds a pick may differ only
between entries the fold error cannot order (the near-tie rule: the oracle's
r at the GPU pick lies within the fold error's slack of the oracle's
maximum). Whatever the picks, steps 8-9 must then be those of the oracle
applied to the GPU's picks: the same candidate intersection, shift, status
and score.
"""
import numpy as np

import oracle.ftm as O

TOL = 1e-5


def normwise(got, want):
    scale = max(1e-30, float(np.abs(want).max()))
    return float(np.abs(np.asarray(got, dtype=np.float64) - want).max()) / scale


def _moduli(ref):
    return [ref["M1"], ref["M2"]]


def _check_steps89(q, res, ref, picks, thm2=False):
    """Steps 8-9 of the oracle on the GPU's picks (equal to ref's when the
    picks agree)."""
    x = O.decode(q.x, q.xdtype, q.N)
    want = O.steps_8_9(x, q.t, picks, _moduli(ref), thm2=thm2)
    assert res["n_cand"] == want["n_cand"], (res, want)
    assert res["shift"] == want["shift"], (res, want)
    assert (res["status"] & 0xFF) == want["status"], (res, want)
    score = float(want["score"])
    assert abs(res["score"] - score) <= 1e-9 * max(1.0, abs(score)), (res["score"], score)


def _same_r(got, want, t):
    """r at a pick: exact for an integral template (integers in fp64), else
    within fp64 rounding of a K-term sum (the two sides add in different
    orders; the oracle may take the FFT route)."""
    if np.all(np.asarray(t) == np.round(t)):
        return got == float(want)
    return abs(got - float(want)) <= 1e-9 * max(1.0, abs(float(want)))


def check_int(b, i, q, res, ref):
    P = b.infos[i]["P"]
    M1, M2, K = ref["M1"], ref["M2"], q.K
    y = b.folds(i).cpu().numpy().astype(np.int64)
    assert np.array_equal(y[:M1 + K - 1], ref["y1"]) and np.array_equal(y[P:P + M2 + K - 1], ref["y2"])
    r = b.corr(i).cpu().numpy().astype(np.float64)
    assert normwise(r[:M1], ref["r1"]) <= TOL and normwise(r[P:P + M2], ref["r2"]) <= TOL
    assert (res["m1"], res["m2"], res["shift"], res["n_cand"]) == (ref["m1"], ref["m2"], ref["shift"], ref["n_cand"])
    assert (res["status"] & 0xFF) == ref["status"]
    assert _same_r(res["score"], ref["score"], q.t)
    assert _same_r(res["r1"], ref["r1"][ref["m1"]], q.t) and _same_r(res["r2"], ref["r2"][ref["m2"]], q.t)


def _picks_real(q, res, ref, slacks):
    """Near-tie rule for the step-7 picks of a real signal; returns True
    when both picks equal the oracle's."""
    exact = True
    for key, mk, rr, slack in (("r1", "m1", ref["r1"], slacks[0]), ("r2", "m2", ref["r2"], slacks[1])):
        m_gpu, m_ref = res[mk], ref[mk]
        if m_gpu != m_ref:
            exact = False
            assert rr[m_gpu] >= rr.max() - slack, (key, m_gpu, m_ref, rr[m_gpu], rr.max(), slack)
        # the rescored value at the pick is the GPU fold's exact correlation
        assert abs(res[key] - rr[m_gpu]) <= slack + TOL * float(np.abs(rr).max()), (key, res[key], rr[m_gpu])
    return exact


def check_real(b, i, q, res, ref, thm2=False):
    """Folds and correlations within 1e-5 normwise; picks by the near-tie
    rule with the slack 2 ||t||_1 max|dy| (the measured fold error); steps
    8-9 those of the oracle on the GPU's picks. Returns True when the
    picks equal the oracle's."""
    P = b.infos[i]["P"]
    M1, M2, K = ref["M1"], ref["M2"], q.K
    y = b.folds(i).cpu().numpy().astype(np.float64)
    assert normwise(y[:M1 + K - 1], ref["y1"]) <= TOL, normwise(y[:M1 + K - 1], ref["y1"])
    assert normwise(y[P:P + M2 + K - 1], ref["y2"]) <= TOL
    r = b.corr(i).cpu().numpy().astype(np.float64)
    assert normwise(r[:M1], ref["r1"]) <= TOL and normwise(r[P:P + M2], ref["r2"]) <= TOL
    t1 = float(np.abs(q.t.astype(np.float64)).sum())
    slacks = []
    for rr, yy, yref in ((ref["r1"], y[:M1 + K - 1], ref["y1"]), (ref["r2"], y[P:P + M2 + K - 1], ref["y2"])):
        slacks.append(2.0 * t1 * float(np.abs(yy - yref).max()) + 1e-9 * float(np.abs(rr).max()))
    exact = _picks_real(q, res, ref, slacks)
    _check_steps89(q, res, ref, [res["m1"], res["m2"]], thm2=thm2)
    return exact


def check_result(q, res, ref, thm2=False):
    """A result without access to the GPU's folds (served requests): +-1
    signals every field exact; real signals the picks by the near-tie rule
    with the slack 2 TOL max|r| (the 1e-5 normwise bar on r) and steps 8-9
    those of the oracle on the GPU's picks. Returns True when the picks
    equal the oracle's."""
    if q.xdtype in ("i8", "bits"):
        assert (res["m1"], res["m2"], res["shift"], res["n_cand"]) == \
            (ref["m1"], ref["m2"], ref["shift"], ref["n_cand"]), (res, ref)
        assert (res["status"] & 0xFF) == ref["status"]
        assert _same_r(res["score"], ref["score"], q.t)
        assert _same_r(res["r1"], ref["r1"][ref["m1"]], q.t) and _same_r(res["r2"], ref["r2"][ref["m2"]], q.t)
        return True
    slacks = [2.0 * TOL * float(np.abs(ref["r1"]).max()), 2.0 * TOL * float(np.abs(ref["r2"]).max())]
    exact = _picks_real(q, res, ref, slacks)
    _check_steps89(q, res, ref, [res["m1"], res["m2"]], thm2=thm2)
    return exact
