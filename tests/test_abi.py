"""Host-side checks of the C ABI (no GPU needed).

- libtm.so loads and exports every function include/tm.h declares;
- the planner (Algorithm 1 step 2) accepts and rejects what the oracle does
  and picks the same moduli;
- the closed-form intersection of steps 8-9 equals the oracle's explicit
  set intersection, exhaustively on small sizes.
"""
import os
import re
import subprocess

import pytest

import oracle.ftm as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def tm():
    from paper_1509_04863_gb300 import _build
    _build.build()
    import paper_1509_04863_gb300 as tm
    tm.lib()
    return tm


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "tm.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tm_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("tm_plan_create", "tm_match", "tm_match_batch", "tm_batch_create", "tm_batch_run"):
        assert required in names


def test_library_exports_every_declared_symbol(tm):
    from paper_1509_04863_gb300 import _build
    out = subprocess.run(["nm", "-D", "--defined-only", _build.LIB], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(tm_\w+)", out))
    missing = [n for n in _declared_functions() if n not in exported]
    assert not missing, missing
    for n in _declared_functions():
        assert getattr(tm.lib(), n) is not None


def test_crt_closed_form_large_values(tm):
    """The closed form at the sizes the library runs (N up to 2^34, moduli
    up to 2^25, residues anywhere), against the intersection counted from
    its definition with Python integers: the naturals v < N with v = m1
    (mod M1) and v = m2 (mod M2) from sympy's Chinese remainder solver, and
    the two wrapped members w_i = m_i + (ceil(N/M_i) - 1) M_i - N tested for
    membership in the other set."""
    import math
    import random
    crt = pytest.importorskip("sympy.ntheory.modular").crt
    rng = random.Random(12345)
    for _ in range(300):
        M1 = rng.randrange(2, 1 << 25)
        M2 = rng.choice([M1 + 1, rng.randrange(2, 1 << 25)])
        if math.gcd(M1, M2) != 1:
            continue
        N = rng.choice([rng.randrange(1, M1 * M2), rng.randrange(M1 * M2, 4 * M1 * M2), rng.randrange(1, 1 << 34)])
        m1, m2 = rng.randrange(M1), rng.randrange(M2)
        v = int(crt([M1, M2], [m1, m2])[0])   # the natural solution in [0, M1 M2)
        nat = [] if v >= N else [v + j * M1 * M2 for j in range(min(3, (N - 1 - v) // (M1 * M2) + 1))]
        n_nat = 0 if v >= N else (N - 1 - v) // (M1 * M2) + 1

        def in_set(w, m, M):
            return w % M == m or w == m + (-(-N // M) - 1) * M - N

        wrapped = set()
        for m, M, mo, Mo in ((m1, M1, m2, M2), (m2, M2, m1, M1)):
            w = m + (-(-N // M) - 1) * M - N
            if 0 <= w and in_set(w, mo, Mo):
                wrapped.add(w)
        want = sorted(set(nat) | wrapped)[:3]
        got = tm.tm_crt_candidates(N, M1, M2, m1, m2, cap=3)
        assert got == want, (N, M1, M2, m1, m2, got, want)
        assert tm.lib().tm_crt_candidates(N, M1, M2, m1, m2, None, 0) == n_nat + len(wrapped), (N, M1, M2, m1, m2)


def test_binding_struct_layouts_match_the_library(tm):
    """The ctypes layouts of the binding have the sizes the compiled
    library gives its public structs (a field added on one side only
    would shift every later field)."""
    import ctypes as C
    structs = [tm.tm_plan_desc, tm.tm_query, tm.tm_result, tm.tm_serve_cfg, tm.tm_result_tagged, tm.tm_serve_stats]
    for which, st in enumerate(structs):
        assert tm.lib().tm_struct_size(which) == C.sizeof(st), (st.__name__, tm.lib().tm_struct_size(which))
    assert tm.lib().tm_struct_size(99) == 0


PLAN_CASES = [
    # N, K, mode, M1, M2, ambig
    (65536, 1024, "paper", 0, 0, False),
    (1 << 24, 4096, "paper", 0, 0, False),
    (1 << 22, 256, "paper", 0, 0, False),      # rejected: 256*257 <= N
    (1 << 22, 256, "paper", 0, 0, True),
    (1 << 24, 300, "auto", 0, 0, False),
    (20000, 100, "auto", 0, 0, False),
    (100, 10, "explicit", 12, 14, False),      # not co-prime
    (100, 10, "explicit", 9, 16, False),       # M1 < K
    (100, 10, "explicit", 11, 13, False),
    (10, 11, "paper", 0, 0, False),            # K > N
    (10, 10, "paper", 0, 0, False),            # M2 = N + 1
    (1, 1, "auto", 0, 0, False),
]


@pytest.mark.parametrize("N,K,mode,M1,M2,ambig", PLAN_CASES)
def test_planner_matches_oracle(tm, N, K, mode, M1, M2, ambig):
    try:
        want = O.plan(N, K, mode, M1, M2, ambig)
    except ValueError:
        want = None
    if want is None:
        with pytest.raises(tm.TMError) as e:
            tm.Plan(N, K, "i8", mode, M1, M2, ambig)
        assert e.value.status == tm.TM_EINVAL
        return
    p = tm.Plan(N, K, "i8", mode, M1, M2, ambig)
    assert (p.info["M1"], p.info["M2"]) == want
    assert p.info["L1"] == -(-N // want[0]) and p.info["L2"] == -(-N // want[1])
    P = p.info["P"]
    assert P >= max(want) + K - 1 and (P & (P - 1)) == 0 and P // 2 < max(want) + K - 1 or P == 1


def test_planner_unsupported_sizes(tm):
    # Table 2's size (N = 2^26, K = 2^16): FFT length 2^17; Fig. 1(a)'s
    # largest template (K = 2^25): 2^26, the longest FFT planned
    assert tm.Plan(1 << 26, 1 << 16, "i8", "paper").info["P"] == 1 << 17
    assert tm.Plan(1 << 26, 1 << 25, "i8", "paper").info["P"] == 1 << 26
    with pytest.raises(tm.TMError) as e:
        tm.Plan(1 << 27, (1 << 25) + 1, "i8", "paper")    # P = 2^27 > 2^26
    assert e.value.status == tm.TM_EUNSUPPORTED


@pytest.mark.parametrize("N,M1,M2", [(19, 4, 5), (30, 5, 6), (31, 5, 7), (50, 7, 8), (20, 6, 7), (85, 9, 10),
                                      (100, 4, 5), (64, 8, 9), (11, 11, 12), (7, 8, 9), (12, 5, 13)])
def test_crt_closed_form_equals_set_intersection(tm, N, M1, M2):
    """Steps 8-9: tm_crt_candidates (closed form, used on the device) lists
    exactly S1 ∩ S2 as the oracle builds it, for every residue pair."""
    for a in range(M1):
        for b in range(M2):
            want = sorted(O.candidate_set(a, M1, N) & O.candidate_set(b, M2, N))
            assert tm.tm_crt_candidates(N, M1, M2, a, b) == want, (N, M1, M2, a, b)


@pytest.mark.parametrize("N,K,mode,M,ambig", [
    (10 ** 6, 64, "paper", (0, 0, 0), True), (10 ** 6, 100, "auto", (0, 0, 0), False),
    (10 ** 6, 63, "paper", (0, 0, 0), False), (5000, 7, "paper", (0, 0, 0), True),
    (10 ** 6, 50, "explicit", (101, 103, 107), False), (10 ** 6, 50, "explicit", (102, 104, 105), False),
    (10 ** 7, 50, "explicit", (51, 52, 53), False), (1 << 20, 16000, "paper", (0, 0, 0), False)])
def test_planner_three_moduli_matches_oracle(tm, N, K, mode, M, ambig):
    """TM_THREE_MODULI against the oracle's plan3 (reading R14): moduli,
    rejection of shared factors and of products not above N, FFT length."""
    try:
        want = O.plan3(N, K, mode, *M, allow_ambig=ambig)
    except ValueError:
        want = None
    if want is None:
        with pytest.raises(tm.TMError) as e:
            tm.Plan(N, K, "i8", mode, M[0], M[1], ambig, three=True, M3=M[2])
        assert e.value.status == tm.TM_EINVAL
        return
    if max(want) + K - 1 > 16384:
        with pytest.raises(tm.TMError) as e:
            tm.Plan(N, K, "i8", mode, M[0], M[1], ambig, three=True, M3=M[2])
        assert e.value.status == tm.TM_EUNSUPPORTED
        return
    p = tm.Plan(N, K, "i8", mode, M[0], M[1], ambig, three=True, M3=M[2])
    assert (p.info["M1"], p.info["M2"], p.info["M3"]) == want
    assert p.info["L3"] == -(-N // want[2])
    P = p.info["P"]
    assert P >= max(want) + K - 1 and P // 2 < max(want) + K - 1
