"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks one oracle function through a route that does not reuse its
code: explicit matrices of Sec. 2-3, brute-force definitions, identities the
theorems state, and the success rates the paper prints (tests/golden/).
A plausible slip in the oracle (a dropped wrap term, convolution instead of
correlation, a wrong index or modulus, a transposed operand) fails at least
one of them.
"""
import math
import os

import numpy as np
import pytest

import oracle.ftm as O
import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            a, b = line.split()
            rows.append((float(a), float(b)))
    return rows


def _pm1(seed, n):
    return W.pm1_signal(W.rng_for(seed), n).astype(np.int64)


# ---------------------------------------------------------------- decoding

def test_decode_bits_lsb_first():
    # byte 0b00000101: bits LSB first = 1,0,1,0,0,0,0,0
    xs = np.array([0b00000101, 0b10000000], dtype=np.uint8)
    got = O.decode(xs, "bits", 10)
    assert got.tolist() == [1, -1, 1, -1, -1, -1, -1, -1, -1, -1]


def test_decode_i8_and_pack_roundtrip():
    x = W.pm1_signal(W.rng_for(3), 1000)
    assert O.decode(x, "i8", 1000).tolist() == x.astype(np.int64).tolist()
    assert O.decode(W.pack_bits(x), "bits", 1000).tolist() == x.astype(np.int64).tolist()


# ---------------------------------------------------------------- step 2

def test_plan_paper_and_auto():
    assert O.plan(65536, 1024, "paper") == (1024, 1025)
    # s(s+1) > N: 256*257 = 65792 > 65536 >= 255*256
    assert O.least_s(65536) == 256
    # 4096*4097 = 16781312 > 2^24 = 16777216 >= 4095*4096 = 16773120
    assert O.least_s(1 << 24) == 4096
    assert O.plan(1 << 24, 300, "auto") == (4096, 4097)
    assert O.plan(1 << 24, 5000, "auto") == (5000, 5001)
    for N in (1, 2, 3, 6, 7, 100, 12345, 999999):
        s = O.least_s(N)
        assert s * (s + 1) > N and (s - 1) * s <= N


def test_plan_rejects():
    with pytest.raises(ValueError):
        O.plan(1 << 22, 256, "paper")          # 256*257 <= 2^22
    assert O.plan(1 << 22, 256, "paper", allow_ambig=True) == (256, 257)
    with pytest.raises(ValueError):
        O.plan(100, 10, "explicit", 12, 14)    # not co-prime
    with pytest.raises(ValueError):
        O.plan(100, 10, "explicit", 9, 16)     # M1 < K
    with pytest.raises(ValueError):
        O.plan(10, 11, "paper")                # K > N


# ---------------------------------------------------------------- step 3

@pytest.mark.parametrize("N,M,K", [(30, 7, 3), (48, 8, 5), (31, 10, 10), (64, 11, 4), (97, 13, 7)])
def test_fold_equals_phi_times_x(N, M, K):
    """y = Phi x with Phi = D_{M+K}(circ(r)), r_k = 1 iff k mod M = 0 (Eq. 3)."""
    x = _pm1(N * 31 + M, N)
    Phi = O.phi_matrix(N, M, M + K - 1)
    assert np.array_equal(O.fold(x, M, K), Phi @ x)
    xr = W.gaussian_signal(W.rng_for(N + M), N).astype(np.float64)
    np.testing.assert_allclose(O.fold(xr, M, K), Phi @ xr, rtol=0, atol=1e-12)


@pytest.mark.parametrize("N,M,K", [(10, 11, 10), (12, 17, 9), (5, 5, 5), (9, 4, 1)])
def test_fold_bruteforce_any_size(N, M, K):
    """Eq. (2) term by term with the (x)_i = (x)_{i mod N} convention, also
    when M > N (a single, wrapping row)."""
    x = _pm1(N + 1000 * M, N)
    L = -(-N // M)
    want = [sum(int(x[(k + i * M) % N]) for i in range(L)) for k in range(M + K - 1)]
    assert O.fold(x, M, K).tolist() == want


# ---------------------------------------------------------------- steps 4-6

@pytest.mark.parametrize("N,M,K", [(60, 7, 5), (97, 11, 7), (128, 16, 16), (50, 13, 2), (33, 40, 30)])
def test_eq4_fold_correlation_identity(N, M, K):
    """r_j = sum_{l < ceil(N/M)} (Tx)_{(j + l M) mod N} for j < M (Eq. (4),
    Thm. 1 with D_{M+K}); (Tx) comes from the brute-force full search."""
    x = _pm1(7 * N + M, N)
    t = _pm1(11 * K + N, K)
    tx = O.full_search_values(x, t)
    L = -(-N // M)
    want = [sum(int(tx[(j + l * M) % N]) for l in range(L)) for j in range(M)]
    r = O.correlate(O.fold(x, M, K), t, M)
    assert r.tolist() == want
    # real-valued signal and template
    xr = W.gaussian_signal(W.rng_for(N), N).astype(np.float64)
    tr = W.gaussian_signal(W.rng_for(K + 5), K).astype(np.float64)
    txr = O.full_search_values(xr, tr)
    wantr = [sum(txr[(j + l * M) % N] for l in range(L)) for j in range(M)]
    np.testing.assert_allclose(O.correlate(O.fold(xr, M, K), tr, M), wantr, rtol=1e-12, atol=1e-10)


@pytest.mark.parametrize("N,M,K", [(40, 9, 4), (64, 16, 8), (90, 12, 12)])
def test_thm1_exchange_with_explicit_matrices(N, M, K):
    """Thm. 1: with That = circ([t 0]) (M x M) and Phi = D_M(circ(r)),
    (That Phi x)_i = (Phi T x)_i for i in [0, M-K]; generically not beyond.
    With D_{M+K} (Sec. 3.2 strategy 1) the match covers every i < M, and it
    equals the oracle's fold + correlation."""
    x = _pm1(N * 3 + K, N)
    t = _pm1(K * 5 + N, K)
    T = O.T_matrix(t, N)
    PhiM = O.phi_matrix(N, M, M)
    That = O.circ(np.concatenate([t, np.zeros(M - K, dtype=np.int64)]))
    lhs = That @ (PhiM @ x)
    rhs = PhiM @ (T @ x)
    assert np.array_equal(lhs[: M - K + 1], rhs[: M - K + 1])
    if N % M == 0:
        # M | N: Phi = [Phi_M ... Phi_M] with Phi_M = I, the Thm. 2 setting,
        # where the exchange holds on every row.
        assert np.array_equal(lhs, rhs)
    elif K > 1:
        assert not np.array_equal(lhs[M - K + 1:], rhs[M - K + 1:])
    PhiMK = O.phi_matrix(N, M, M + K)
    ThatK = O.circ(np.concatenate([t, np.zeros(M, dtype=np.int64)]))
    lhsK = ThatK @ (PhiMK @ x)
    rhsK = PhiMK @ (T @ x)
    assert np.array_equal(lhsK[:M], rhsK[:M])
    assert O.correlate(O.fold(x, M, K), t, M).tolist() == rhsK[:M].tolist()


@pytest.mark.parametrize("M,K", [(7, 3), (64, 17), (1025, 1024), (300, 299)])
def test_fft_correlation_equals_direct_sum(M, K):
    """Steps 4-6 (FFT route, with the conjugate) equal the direct sum."""
    y = _pm1(M * K, M + K - 1) * 3
    t = _pm1(M + K, K)
    r_direct = O.correlate(y, t, M)
    r_fft = O.correlate_fft(y, t, M)
    assert np.max(np.abs(r_fft - r_direct)) < 1e-6
    # a pure-Python loop on the smallest case
    if M * K < 5000:
        want = [sum(int(t[i]) * int(y[j + i]) for i in range(K)) for j in range(M)]
        assert r_direct.tolist() == want


def test_convolution_reading_fails_on_planted_window():
    """Reading R3: Algorithm 1 step 6 printed without a conjugate would
    convolve; with a planted window only the correlating route peaks at the
    planted position."""
    N, K = 4096, 256
    x = _pm1(77, N)
    k = 1234
    t = x[(np.arange(K) + k) % N]
    M = K
    y = O.fold(x, M, K)
    r = O.correlate(y, t, M)
    assert O.argmax_first(r) == k % M
    P = 1 << (M + K - 2).bit_length()
    conv = np.fft.ifft(np.fft.fft(t, P) * np.fft.fft(np.pad(y, (0, P - y.size)))).real[:M]
    assert int(np.argmax(conv)) != k % M


# ---------------------------------------------------------------- step 7

def test_argmax_first_ties():
    assert O.argmax_first(np.array([1, 5, 5, 2])) == 1
    assert O.argmax_first(np.array([7])) == 0
    assert O.argmax_first(np.array([-3.0, -1.0, -1.0])) == 1


# ---------------------------------------------------------------- steps 8-9

@pytest.mark.parametrize("M1,M2,N", [(4, 5, 19), (5, 6, 30), (7, 8, 50), (6, 7, 20), (9, 10, 85)])
def test_crt_recovers_every_shift_exhaustive(M1, M2, N):
    """Thm. 4: a shift m in [0, N) is recovered from its exact residues
    m mod M1, m mod M2. Intersection members other than m can only be the
    wrapped candidates (m~_i + (L_i-1) M_i) - N of Alg. 1 step 8 (R5)."""
    L1, L2 = -(-N // M1), -(-N // M2)
    for m in range(N):
        S1 = O.candidate_set(m % M1, M1, N)
        S2 = O.candidate_set(m % M2, M2, N)
        I = S1 & S2
        assert m in I
        wrapped = {(m % M1) + (L1 - 1) * M1 - N, (m % M2) + (L2 - 1) * M2 - N}
        assert I - {m} <= wrapped
    # exhaustive over all residue pairs: every intersection member is
    # congruent to both residues or is a wrapped candidate
    for a in range(M1):
        for b in range(M2):
            I = O.candidate_set(a, M1, N) & O.candidate_set(b, M2, N)
            for m in I:
                assert (m % M1 == a or m == a + (L1 - 1) * M1 - N)
                assert (m % M2 == b or m == b + (L2 - 1) * M2 - N)


def test_candidate_set_size_and_membership():
    # ceil(95/10) = 10 members; 3 + 9*10 = 93 < 95 needs no wrap
    assert O.candidate_set(3, 10, 95) == {3 + 10 * i for i in range(10)}
    # 7 + 9*10 = 97 wraps to 97 - 95 = 2
    assert O.candidate_set(7, 10, 95) == {7 + 10 * i for i in range(9)} | {2}


# ---------------------------------------------------------------- full search & planted shift

def test_noiseless_planted_tx_equals_K_and_full_search():
    """Sec. 3.5: with t = [x_m .. x_{m+K-1}], (Tx)_m = K; the full search
    returns m when the maximum is unique."""
    N, K = 2048, 64
    for seed in range(5):
        q = W.planted_query(seed, N, K)
        x = O.decode(q.x, "i8", N)
        t = O.template_values(q.t)
        tx = O.full_search_values(x, t)
        assert tx[q.k_star] == K
        assert O.full_search(x, t) == q.k_star
        assert np.array_equal(O.full_search_fft(x, t), tx)


def test_ftm_single_config_recovers_or_fails_consistently():
    """Config-1 shape: N = 65536, K = 1024, M = 1024/1025. Whenever the step-7
    residues equal k* mod M_i, the recovered shift is k* (Thm. 4)."""
    hits = 0
    for seed in range(6):
        q = W.single_query(seed)
        res = O.match_query(q)
        k = q.k_star
        if res["m1"] == k % 1024 and res["m2"] == k % 1025:
            assert res["shift"] == k and res["status"] == O.FOUND
            hits += 1
        else:
            assert res["shift"] != k or res["status"] == O.RESOLVED
    assert hits >= 1


# ---------------------------------------------------------------- Thm. 3

def test_thm3_sufficient_condition_on_barker_inputs():
    """Thm. 3: if (Tx)_m / (2 ceil(N/M) + 1) > max_{k != m} (Tx)_k then the
    true position is among the candidates of step 8 (m = m~ mod M). The
    Barker-13 template has aperiodic sidelobes of magnitude <= 1."""
    with open(os.path.join(GOLDEN, "barker13.txt")) as f:
        b = [int(v) for line in f if not line.startswith("#") for v in line.split()]
    t = np.array(b, dtype=np.int64)
    K = t.size
    for M1, N in ((13, 39), (14, 52), (13, 65)):
        M2 = M1 + 1
        for m in range(N):
            x = np.zeros(N, dtype=np.int64)
            x[(np.arange(K) + m) % N] = t
            tx = O.full_search_values(x, t)
            assert O.thm3_condition(tx, m, M1)
            res = O.ftm(x, t, M1, M2)
            assert res["m1"] == m % M1
            if O.thm3_condition(tx, m, M2):
                assert res["m2"] == m % M2


# ---------------------------------------------------------------- Thm. 5 and Tables 1-2

def _fold_fail_rate(N, K, M, n, seed0):
    fails = 0
    for s in range(n):
        q = W.planted_query(seed0 + s, N, K)
        x = O.decode(q.x, "i8", N)
        t = O.template_values(q.t)
        r = O.correlate_fft(O.fold(x, M, K), t, M)
        if O.argmax_first(np.rint(r)) != q.k_star % M:
            fails += 1
    return fails / n


def test_thm5_bound_dominates_empirical_failure():
    """Per-modulus failure probability <= M e^{-K/(8L)} + 4(L-1)/K (Thm. 5)."""
    N, K = 1 << 16, 2048
    bound = O.thm5_fold_failure_bound(N, K, K)
    assert bound < 1
    assert _fold_fail_rate(N, K, K, 30, 4242) <= bound


def _binom_two_sided_p(k, n, p):
    """Exact two-sided binomial p-value (sum of outcomes no likelier than k)."""
    pmf = [math.comb(n, i) * p ** i * (1 - p) ** (n - i) for i in range(n + 1)]
    pk = pmf[k]
    return min(1.0, sum(v for v in pmf if v <= pk * (1 + 1e-9)))


def _success_rate(N, K, n, seed0, snr=None):
    ok = 0
    for s in range(n):
        q = W.planted_query(seed0 + s, N, K) if snr is None else W.snr_query(seed0 + s, N, K, snr)
        x = O.decode(q.x, q.xdtype, N)
        t = O.template_values(q.t)
        res = O.ftm(x, t, K, K + 1, corr="fft")
        ok += int(res["shift"] == q.k_star)
    return ok


@pytest.mark.parametrize("log2N,n", [(23, 12), (24, 12), (25, 8)])
def test_table1_success_rates(log2N, n):
    """Table 1 (Sec. 4), K = N/2^10: the oracle's success count is consistent
    with the printed probability (exact binomial test, p > 0.001)."""
    table = dict(_read_table("table1_success.txt"))
    p = table[log2N]
    N = 1 << log2N
    k = _success_rate(N, N >> 10, n, 9000 + log2N * 100)
    assert _binom_two_sided_p(k, n, p) > 1e-3, (log2N, k, n, p)


@pytest.mark.parametrize("snr,n", [(20.0, 3), (-6.0, 3)])
def test_table2_success_rates(snr, n):
    """Table 2 (Sec. 4), N = 2^26, K = 2^16, Gaussian noise on x (R8)."""
    table = dict(_read_table("table2_success.txt"))
    p = table[snr]
    k = _success_rate(1 << 26, 1 << 16, n, 77000 + int(snr * 10), snr=snr)
    pp = min(max(p, 1e-3), 1 - 1e-3)
    assert _binom_two_sided_p(k, n, pp) > 1e-3, (snr, k, n, p)


# ---------------------------------------------------------------------------
# Slices of one signal: Eq. (2) and Eq. (1) are sums over the entries of x,
# so restricting them to the pieces of any partition and adding the pieces
# must give the whole (checked against fold() and tx_at(), which never
# restrict); the single piece [0, N) is the whole.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N,M,K", [(1000, 37, 20), (4096, 64, 65), (777, 800, 50), (5000, 71, 70)])
def test_fold_slices_add_up(N, M, K):
    rng = np.random.default_rng(N + M)
    x = rng.integers(-3, 4, N).astype(np.int64)
    want = O.fold(x, M, K)
    assert np.array_equal(O.fold_slice(x, 0, N, M, K), want)
    for _ in range(5):
        cuts = np.sort(rng.choice(np.arange(1, N), size=int(rng.integers(1, 6)), replace=False))
        bounds = [0, *cuts.tolist(), N]
        got = sum(O.fold_slice(x[a:b], a, N, M, K) for a, b in zip(bounds[:-1], bounds[1:]))
        assert np.array_equal(got, want)


def test_score_slices_add_up():
    rng = np.random.default_rng(5)
    N, K = 3001, 257
    x = rng.integers(-1, 2, N).astype(np.int64) * 2 + 1
    t = rng.integers(-2, 3, K).astype(np.int64)
    for m in (0, 5, N - 100, N - 1):
        want = O.tx_at(x, t, m)
        bounds = [0, 1000, 1016, 2990, N]
        got = sum(O.tx_slice(x[a:b], a, N, t, m) for a, b in zip(bounds[:-1], bounds[1:]))
        assert got == want
        assert O.tx_slice(x, 0, N, t, m) == want


# ---------------------------------------------------------------------------
# Thm. 2 (the second sampling matrix): fold_thm2 against Phi = [I ... I]
# built as a matrix; the theorem's identity T^ Phi x = Phi T_bar x with the
# block-diagonal T_bar, from explicit matrices; the circular correlation by
# an FFT of length M; a window inside one block reads the true (Tx)_m.
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("N,M,K", [(60, 12, 5), (61, 12, 5), (100, 7, 7), (128, 32, 9)])
def test_thm2_fold_and_identity(N, M, K):
    rng = np.random.default_rng(N * M)
    x = rng.integers(-5, 6, N).astype(np.int64)
    t = rng.integers(-3, 4, K).astype(np.int64)
    L = -(-N // M)
    xp = np.concatenate([x, np.zeros(L * M - N, dtype=np.int64)])
    Phi = np.hstack([np.eye(M, dtype=np.int64)] * L)
    y = O.fold_thm2(x, M)
    assert np.array_equal(y, Phi @ xp)
    tM = np.concatenate([t, np.zeros(M - K, dtype=np.int64)])
    That = O.circ(tM)
    Tbar = np.kron(np.eye(L, dtype=np.int64), That)
    assert np.array_equal(That @ (Phi @ xp), Phi @ (Tbar @ xp))
    r = O.correlate_circular(y, t, M)
    assert np.array_equal(r, That @ y)
    rf = np.real(np.fft.ifft(np.conj(np.fft.fft(tM)) * np.fft.fft(y)))
    assert np.allclose(rf, r)


def test_thm2_window_inside_a_block():
    rng = np.random.default_rng(3)
    N, M, K = 4096, 256, 64
    x = np.where(rng.random(N) < 0.5, 1, -1).astype(np.int64)
    k_star = 5 * M + 100                     # the window [k*, k*+K) stays in block 5
    t = x[k_star:k_star + K].copy()
    L = N // M
    blocks = x.reshape(L, M)
    # block-diagonal correlation at k* mod M, block 5 alone, equals (Tx)_{k*} = K
    tM = np.concatenate([t, np.zeros(M - K, dtype=np.int64)])
    assert int((O.circ(tM) @ blocks[5])[k_star % M]) == O.tx_at(x, t, k_star) == K
    # and the whole Thm. 2 fold correlation is the sum of the blocks' terms
    r = O.correlate_circular(O.fold_thm2(x, M), t, M)
    assert r[k_star % M] == sum(int((O.circ(tM) @ b)[k_star % M]) for b in blocks)
    assert k_star in O.candidate_set_thm2(k_star % M, M, N)
    assert all(v < N for v in O.candidate_set_thm2(M - 1, M, N - 3))


# ---------------------------------------------------------------------------
# Thm. 4 with three moduli: the intersection of the three candidate sets is
# checked exhaustively against the CRT (every shift of small signals is
# recovered, and only it when M1 M2 M3 >= N); the chosen moduli are pairwise
# co-prime and reach N; three moduli recover a planted shift where K(K+1) <= N
# leaves two moduli ambiguous.
# ---------------------------------------------------------------------------

def test_three_moduli_crt_exhaustive():
    for (M1, M2, M3) in [(3, 4, 5), (5, 6, 7), (7, 8, 9)]:
        for N in (M1 * M2 * M3 - 5, M1 * M2 * M3, M1 * M2 * M3 + 9):
            for m in range(0, N, max(1, N // 37)):
                Ss = [O.candidate_set(m % M, M, N) for M in (M1, M2, M3)]
                I = set.intersection(*Ss)
                assert m in I
                if M1 * M2 * M3 >= N:
                    # naturals are unique mod M1 M2 M3 (Thm. 4); any other
                    # member is the wrapped member of one of the sets
                    nat = [v for v in I if v % M1 == m % M1 and v % M2 == m % M2 and v % M3 == m % M3]
                    assert nat == [m]
                    wrapped = {m % M + (-(-N // M) - 1) * M - N for M in (M1, M2, M3)}
                    assert all(v == m or v in wrapped for v in I)


@pytest.mark.parametrize("N,K,mode", [(10 ** 6, 64, "paper"), (10 ** 6, 100, "auto"), (5000, 7, "paper")])
def test_three_moduli_plan(N, K, mode):
    M1, M2, M3 = O.plan3(N, K, mode, allow_ambig=True)
    assert min(M1, M2, M3) >= K and M1 % 2 == 1
    assert math.gcd(M1, M2) == math.gcd(M1, M3) == math.gcd(M2, M3) == 1
    if mode == "auto":
        assert M1 * M2 * M3 > N


def test_three_moduli_recover_where_two_are_ambiguous():
    # a strong planted window in weak noise, so that step 7 succeeds for
    # every modulus although K (K+1) = 66306 < N: two moduli then leave
    # several members of S1 ∩ S2, three leave exactly the planted shift
    rng = np.random.default_rng(8)
    N, K = 300000, 257
    x = 0.01 * rng.standard_normal(N)
    k_star = 123457
    t = np.where(rng.random(K) < 0.5, 1.0, -1.0)
    x[(np.arange(K) + k_star) % N] = t
    two = O.ftm(x, t, K, K + 1)
    assert two["m1"] == k_star % K and two["m2"] == k_star % (K + 1)
    assert two["n_cand"] > 1 and k_star in two["I"]
    M1, M2, M3 = O.plan3(N, K, "paper", allow_ambig=True)   # 257 * 258 * 259 > N
    assert M1 * M2 * M3 > N
    three = O.ftm_multi(x, t, (M1, M2, M3))
    assert three["n_cand"] == 1 and three["shift"] == k_star and three["status"] == O.FOUND


# ---------------------------------------------------------------------------
# Steps 7-9 assembled end to end, recomputed without the oracle's helpers:
# (Tx)_k by brute force, r_j by Eq. (4) (Alg. 1) or by the explicit circ([t 0])
# product (Thm. 2), the argmax by a Python loop, the candidate sets by
# listing their members, and step 9 (reading R6: the largest exact (Tx)_m
# over the intersection, ties to the smallest m).
# ---------------------------------------------------------------------------

def _brute_tx(x, t):
    N, K = len(x), len(t)
    return [sum(int(t[i]) * int(x[(k + i) % N]) for i in range(K)) for k in range(N)]


def _first_argmax(v):
    best, arg = None, -1
    for j, val in enumerate(v):
        if best is None or val > best:
            best, arg = val, j
    return arg


def _step9(I, tx):
    if not I:
        return -1, O.EMPTY
    if len(I) == 1:
        return I[0], O.FOUND
    best = max(tx[m] for m in I)
    return min(m for m in I if tx[m] == best), O.RESOLVED


def _expected_alg1(x, t, M1, M2):
    N = len(x)
    tx = _brute_tx(x, t)
    out = {}
    sets = []
    for key, M in (("m1", M1), ("m2", M2)):
        L = -(-N // M)
        r = [sum(tx[(j + l * M) % N] for l in range(L)) for j in range(M)]   # Eq. (4)
        m = _first_argmax(r)
        out[key] = m
        members = set()
        for l in range(L):
            members.add((m + l * M) % N)
        sets.append(members)
    I = sorted(v for v in sets[0] if v in sets[1])
    out["I"] = I
    out["shift"], out["status"] = _step9(I, tx)
    return out, tx


def _check_against(res, want):
    assert res["m1"] == want["m1"] and res["m2"] == want["m2"]
    assert res["I"] == want["I"]
    assert res["n_cand"] == len(want["I"])
    assert res["shift"] == want["shift"] and res["status"] == want["status"]


def test_step9_resolution_by_largest_exact_score():
    """Alg. 1 steps 7-9 with M1 M2 <= N (several members of S1 ∩ S2): the
    oracle's shift is the member with the largest (Tx)_m, and instances exist
    where that is not the smallest member (a rule 'smallest m' fails here)."""
    not_smallest = resolved = 0
    for seed in range(60):
        rng = np.random.default_rng(10_000 + seed)
        M1 = int(rng.integers(3, 7))
        M2 = M1 + 1
        N = int(rng.integers(4, 9)) * M1 * M2 + int(rng.integers(0, M1))
        K = int(rng.integers(2, M1 + 1))
        x = np.where(rng.random(N) < 0.5, 1, -1).astype(np.int64)
        k_star = int(rng.integers(0, N))
        t = x[(np.arange(K) + k_star) % N].copy()
        want, tx = _expected_alg1(x, t, M1, M2)
        res = O.ftm(x, t, M1, M2)
        _check_against(res, want)
        if want["status"] == O.RESOLVED:
            resolved += 1
            if want["shift"] != want["I"][0]:
                not_smallest += 1
            assert res["score"] == tx[want["shift"]]
    assert resolved >= 10 and not_smallest >= 3, (resolved, not_smallest)


def test_step9_ties_go_to_smallest_member():
    """x periodic with period M1 M2 makes (Tx)_m equal on every member of
    S1 ∩ S2 (they differ by multiples of M1 M2): step 9 then returns the
    smallest one (reading R6). Checked for Alg. 1 (ftm, three-moduli
    ftm_multi with a period of M1 M2 M3) and the Thm. 2 variant."""
    for M1, reps, seed in ((4, 5, 1), (5, 3, 2), (3, 7, 3)):
        M2 = M1 + 1
        rng = np.random.default_rng(seed)
        period = np.where(rng.random(M1 * M2) < 0.5, 1, -1).astype(np.int64)
        x = np.tile(period, reps)
        N = x.size
        K = M1
        t = x[(np.arange(K) + 7) % N].copy()
        want, tx = _expected_alg1(x, t, M1, M2)
        res = O.ftm(x, t, M1, M2)
        _check_against(res, want)
        assert len(want["I"]) == reps and want["status"] == O.RESOLVED
        assert len({tx[m] for m in want["I"]}) == 1
        assert res["shift"] == want["I"][0]
        # Thm. 2 variant: M1 M2 divides N, so there is no padding and the
        # members below N are the same naturals
        r2 = O.ftm_thm2(x, t, M1, M2)
        if r2["n_cand"] > 1:
            assert r2["shift"] == min(r2["I"]) and r2["status"] == O.RESOLVED
    Ms = (3, 4, 5)
    rng = np.random.default_rng(9)
    x = np.tile(np.where(rng.random(60) < 0.5, 1, -1).astype(np.int64), 4)
    t = x[(np.arange(3) + 11) % x.size].copy()
    res = O.ftm_multi(x, t, Ms)
    if res["n_cand"] > 1:
        tx = _brute_tx(x, t)
        assert len({tx[m] for m in res["I"]}) == 1
        assert res["shift"] == res["I"][0] and res["status"] == O.RESOLVED


@pytest.mark.parametrize("N,M1,K", [(60, 5, 3), (61, 5, 3), (47, 4, 4), (90, 9, 5), (35, 6, 6)])
def test_ftm_thm2_assembled_from_explicit_matrices(N, M1, K):
    """ftm_thm2 (Thm. 2 sampling, reading R13) against its definition built
    by hand: y = [I_M ... I_M] x' (x zero-padded to a multiple of M), r =
    circ([t 0_{M-K}]) y, m~ by a Python loop, candidates m~ + l M below N
    listed one by one, intersection, step 9 by the brute-force (Tx)_m.
    Covers M | N and M not dividing N, planted windows and random ones."""
    M2 = M1 + 1
    for seed in range(8):
        rng = np.random.default_rng(N * 100 + M1 * 10 + seed)
        x = np.where(rng.random(N) < 0.5, 1, -1).astype(np.int64)
        k_star = int(rng.integers(0, N))
        t = x[(np.arange(K) + k_star) % N].copy()
        if seed % 2:
            t[int(rng.integers(0, K))] *= -1
        tx = _brute_tx(x, t)
        want = {}
        sets = []
        for key, M in (("m1", M1), ("m2", M2)):
            L = -(-N // M)
            xp = np.concatenate([x, np.zeros(L * M - N, dtype=np.int64)])
            Phi = np.hstack([np.eye(M, dtype=np.int64)] * L)
            y = Phi @ xp
            C = np.array([[t[(c - r) % M] if (c - r) % M < K else 0 for c in range(M)] for r in range(M)],
                         dtype=np.int64)
            r = C @ y
            m = _first_argmax(r.tolist())
            want[key] = m
            s = []
            l = 0
            while m + l * M < N:
                s.append(m + l * M)
                l += 1
            sets.append(set(s))
        I = sorted(sets[0] & sets[1])
        shift, status = _step9(I, tx)
        res = O.ftm_thm2(x, t, M1, M2)
        assert res["m1"] == want["m1"] and res["m2"] == want["m2"]
        assert res["I"] == I and res["n_cand"] == len(I)
        assert res["shift"] == shift and res["status"] == status
        assert res["score"] == (tx[shift] if shift >= 0 else 0)


def test_thm3_condition_rejects_when_hypothesis_fails():
    """Thm. 3's hypothesis (reading R10: the printed factor 1/(2L+1)): true
    only when (Tx)_m / (2L + 1) exceeds every other (Tx)_k; here N = 10,
    M = 5, L = 2, so the factor is 1/5."""
    base = np.array([3, 1, 0, -2, 12, 1, 2, 0, 3, -1], dtype=np.int64)
    assert not O.thm3_condition(base, 4, 5)        # 12/5 = 2.4 < 3 (true with 1/(2L-1) = 1/3)
    hi = base.copy()
    hi[4] = 16
    assert O.thm3_condition(hi, 4, 5)              # 16/5 = 3.2 > 3
    eq = base.copy()
    eq[4] = 15
    assert not O.thm3_condition(eq, 4, 5)          # 15/5 = 3: not strictly above
    assert not O.thm3_condition(hi, 0, 5)          # m not the peak


def test_thm5_bound_values():
    """Thm. 5's per-modulus bound M e^{-K/(8L)} + 4(L-1)/K at values worked
    out by hand: N = 2^16, K = M = 2048 gives L = 32, 2048 e^{-8} + 124/2048
    = 0.687027 + 0.060547; N = 2^20, K = M = 2^16 gives L = 16,
    65536 e^{-512} + 60/65536."""
    assert O.thm5_fold_failure_bound(1 << 16, 2048, 2048) == pytest.approx(0.7475744, rel=1e-6)
    assert O.thm5_fold_failure_bound(1 << 20, 1 << 16, 1 << 16) == pytest.approx(60 / 65536, rel=1e-9)
    # L = 1 (M >= N): no mixing term
    assert O.thm5_fold_failure_bound(100, 100, 100) == pytest.approx(100 * math.exp(-12.5), rel=1e-12)
