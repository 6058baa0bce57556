"""CPU oracle for Algorithm 1 (FTM) of Hsieh, Lu & Pei, "Fast Template
Matching by Subsampled Circulant Matrix" (arXiv 1509.04863).

TEST INFRASTRUCTURE. Only the tests, the entry module's smoke() check and the
benchmark's CPU-baseline leg may import this module. The CUDA library never
calls it and shares no code, table or helper with it.

Plain, slow and direct: integers are kept in int64 and reals in float64;
each step follows the paper's order and notation. Library primitives
(np.correlate, np.fft) serve only as single steps.

Readings taken where the paper is silent, garbled or inconsistent (each is
listed again in the design notes):
  R1 (Eq. 1, Sec. 3.5)  shifts are searched over 0 <= k < N (k = 0 included).
  R2 (Alg. 1 step 3)    the fold is indexed modulo N (Sec. 2 notation), for
                        k = 0 .. M+K-2; the extra entry k = M+K-1 is unused.
  R3 (Alg. 1 step 6)    the product uses conj(FFT(t)): cross-correlation, as
                        (Tx)_k in Sec. 3 defines it, not convolution.
  R4 (Alg. 1 step 7)    the argmax runs over j = 0 .. M-1 (Sec. 3.3 uses k < M);
                        ties go to the smallest j.
  R5 (Alg. 1 step 8)    candidate positions are reduced modulo N.
  R6 (Alg. 1 step 9)    an empty intersection returns shift -1 (EMPTY); more
                        than one element is resolved by the largest exact
                        (Tx)_m, ties to the smallest m (RESOLVED).
  R7 (Alg. 1 step 2)    mode "paper" uses M1 = K, M2 = K+1 (Sec. 3.5, Sec. 4);
                        mode "auto" uses M1 = max(K, s), M2 = M1+1 with s the
                        least integer such that s(s+1) > N.
  R8 (Sec. 4, Table 2)  SNR = 10 log10(E[x^2] / s^2) with noise on x only.
  R14 (Thm. 4)          three moduli: consecutive integers c, c+1, c+2 from
                        the least odd c >= K (PAPER) or >= max(K, s) with
                        s(s+1)(s+2) > N (AUTO), pairwise co-prime.
  R13 (Thm. 2)          the second sampling matrix uses Phi_M = I_M on x
                        zero-padded to a multiple of M, a circular correlation
                        of period M, and candidate positions below N only.
"""
from __future__ import annotations

import math
from typing import Dict, Iterable, List, Set, Tuple

import numpy as np

FOUND, EMPTY, RESOLVED = 0, 1, 2
STATUS_NAMES = {FOUND: "FOUND", EMPTY: "EMPTY", RESOLVED: "RESOLVED"}


# ---------------------------------------------------------------------------
# Input decoding (storage -> mathematical values)
# ---------------------------------------------------------------------------

def decode(xs: np.ndarray, xdtype: str, N: int) -> np.ndarray:
    """Signal values x_0 .. x_{N-1}: int64 for +-1 codes, float64 for reals."""
    if xdtype == "i8":
        v = xs[:N].astype(np.int64)
        return np.where(v < 0, -1, 1).astype(np.int64)
    if xdtype == "bits":
        b = np.unpackbits(xs.astype(np.uint8), bitorder="little")[:N].astype(np.int64)
        return 2 * b - 1
    if xdtype in ("f16", "f32"):
        return xs[:N].astype(np.float64)
    raise ValueError(f"unknown dtype {xdtype}")


def template_values(t: np.ndarray) -> np.ndarray:
    """Template as int64 when every entry is an integer, else float64."""
    t64 = np.asarray(t, dtype=np.float64)
    if np.all(t64 == np.round(t64)) and np.all(np.abs(t64) < 2 ** 31):
        return t64.astype(np.int64)
    return t64


# ---------------------------------------------------------------------------
# Step 2: choice of the co-prime moduli (Alg. 1 step 2; Sec. 3.5 proof of
# Thm. 5 "M1 = K and M2 = K+1"; Sec. 4 testing procedure).
# ---------------------------------------------------------------------------

def least_s(N: int) -> int:
    """Least integer s with s(s+1) > N."""
    s = max(1, int(math.isqrt(N)) - 1)
    while s * (s + 1) <= N:
        s += 1
    while s > 1 and (s - 1) * s > N:
        s -= 1
    return s


def plan(N: int, K: int, mode: str = "paper", M1: int = 0, M2: int = 0,
         allow_ambig: bool = False) -> Tuple[int, int]:
    """Moduli (M1, M2) per Alg. 1 step 2; raises ValueError when invalid."""
    if K < 1 or N < 1 or K > N:
        raise ValueError("need 1 <= K <= N")
    if mode == "paper":
        M1, M2 = K, K + 1
    elif mode == "auto":
        M1 = max(K, least_s(N))
        M2 = M1 + 1
    elif mode == "explicit":
        pass
    else:
        raise ValueError(mode)
    if M1 < K or M2 < K:
        raise ValueError("step 2 needs M1 >= K and M2 >= K")
    if math.gcd(M1, M2) != 1:
        raise ValueError("step 2 needs co-prime M1, M2")
    if M1 * M2 <= N and not allow_ambig:
        raise ValueError("step 2 needs M1*M2 > N (pass allow_ambig to accept)")
    return M1, M2


# ---------------------------------------------------------------------------
# Step 3: downsampling (Alg. 1 step 3; Eq. (2); Phi = D_{M+K}(circ(r)) from
# Eq. (3) with the D_{M+K} strategy of Sec. 3.2).
# ---------------------------------------------------------------------------

def ceil_div(a: int, b: int) -> int:
    return -(-a // b)


def fold(x: np.ndarray, M: int, K: int) -> np.ndarray:
    """(y_M)_k = sum_{i=0}^{ceil(N/M)-1} x_{(k + i M) mod N}, k = 0..M+K-2."""
    N = x.shape[0]
    L = ceil_div(N, M)
    k = np.arange(M + K - 1, dtype=np.int64)
    y = np.zeros(M + K - 1, dtype=x.dtype)
    for i in range(L):
        y += x[(k + i * M) % N]
    return y


def fold_slice(xs: np.ndarray, n0: int, N: int, M: int, K: int) -> np.ndarray:
    """Eq. (2) keeping only the terms whose index lies in the slice
    [n0, n0 + len(xs)) of a length-N signal (xs = x_{n0} .. x_{n0+len-1}):
    (y_M)_k = sum_{i<L} x_{(k+iM) mod N} [n0 <= (k+iM) mod N < n0+len]."""
    n1 = n0 + xs.shape[0]
    L = ceil_div(N, M)
    k = np.arange(M + K - 1, dtype=np.int64)
    y = np.zeros(M + K - 1, dtype=xs.dtype)
    for i in range(L):
        idx = (k + i * M) % N
        inside = (idx >= n0) & (idx < n1)
        y[inside] += xs[idx[inside] - n0]
    return y


# ---------------------------------------------------------------------------
# Steps 4-6: fast correlation in the low-dimensional space. Its result is
# r_j = sum_{i<K} t_i y_{j+i} for j < M (Thm. 1 with D_{M+K}); the paper
# computes it by FFT (steps 5-6, reading R3).
# ---------------------------------------------------------------------------

def correlate(y: np.ndarray, t: np.ndarray, M: int) -> np.ndarray:
    """Direct sum r_j = sum_{i<K} t_i y_{j+i}, j = 0..M-1 (exact for ints)."""
    K = t.shape[0]
    assert y.shape[0] >= M + K - 1
    dt = np.int64 if (y.dtype.kind == "i" and t.dtype.kind == "i") else np.float64
    return np.correlate(y[:M + K - 1].astype(dt), t.astype(dt), mode="valid")[:M]


def correlate_fft(y: np.ndarray, t: np.ndarray, M: int, P: int = 0) -> np.ndarray:
    """Steps 4-6 as printed, with conj(FFT(t_M)) (R3), in float64.

    t_M = [t 0] and y are zero-padded to a common length P >= M+K-1 so the
    circular product equals the linear correlation on j < M."""
    K = t.shape[0]
    need = M + K - 1
    if P < need:
        P = 1 << (need - 1).bit_length()
    yp = np.zeros(P)
    yp[:need] = y[:need]
    tp = np.zeros(P)
    tp[:K] = t
    r = np.fft.ifft(np.conj(np.fft.fft(tp)) * np.fft.fft(yp))
    return r.real[:M]


# ---------------------------------------------------------------------------
# Step 7: matching position (Alg. 1 step 7, Sec. 3.3 with k < M; R4).
# ---------------------------------------------------------------------------

def argmax_first(r: np.ndarray) -> int:
    m = r.max()
    return int(np.flatnonzero(r == m)[0])


# ---------------------------------------------------------------------------
# Steps 8-9: candidate sets and their intersection (Alg. 1 steps 8-9, Thm. 4).
# ---------------------------------------------------------------------------

def candidate_set(m_tilde: int, M: int, N: int) -> Set[int]:
    """S_M = {(m~ + i M) mod N : i = 0 .. ceil(N/M)-1} (R5)."""
    L = ceil_div(N, M)
    return {int((m_tilde + i * M) % N) for i in range(L)}


def tx_at(x: np.ndarray, t: np.ndarray, m: int):
    """(Tx)_m = sum_{i<K} t_i x_{(m+i) mod N} (Sec. 3)."""
    N = x.shape[0]
    K = t.shape[0]
    idx = (np.arange(K, dtype=np.int64) + m) % N
    if x.dtype.kind == "i" and t.dtype.kind == "i":
        return int(np.dot(t, x[idx]))
    return float(np.dot(t.astype(np.float64), x[idx].astype(np.float64)))


def tx_slice(xs: np.ndarray, n0: int, N: int, t: np.ndarray, m: int):
    """(Tx)_m keeping only the terms whose index lies in the slice
    [n0, n0 + len(xs)) of a length-N signal."""
    K = t.shape[0]
    idx = (np.arange(K, dtype=np.int64) + m) % N
    inside = (idx >= n0) & (idx < n0 + xs.shape[0])
    if xs.dtype.kind == "i" and t.dtype.kind == "i":
        return int(np.dot(t[inside], xs[idx[inside] - n0]))
    return float(np.dot(t[inside].astype(np.float64), xs[idx[inside] - n0].astype(np.float64)))


def intersect_and_resolve(x: np.ndarray, t: np.ndarray, sets: List[Set[int]]) -> Dict:
    """Alg. 1 step 9 on the candidate sets of step 8 (R6): their
    intersection I; |I| = 1 gives the shift (FOUND), |I| = 0 gives -1
    (EMPTY), |I| > 1 the member with the largest exact (Tx)_m, ties to the
    smallest m (RESOLVED); score = (Tx)_shift (0 without a shift)."""
    I = sorted(set.intersection(*sets))
    if len(I) == 0:
        shift, status = -1, EMPTY
    elif len(I) == 1:
        shift, status = I[0], FOUND
    else:
        scores = [tx_at(x, t, m) for m in I]
        shift, status = I[scores.index(max(scores))], RESOLVED
    score = tx_at(x, t, shift) if shift >= 0 else 0
    return dict(I=I, shift=int(shift), status=status, n_cand=len(I), score=score)


def steps_8_9(x: np.ndarray, t: np.ndarray, picks, moduli, thm2: bool = False) -> Dict:
    """Steps 8-9 for given step-7 maxima m~_j of the moduli M_j: candidate
    sets (candidate_set, or candidate_set_thm2 for the Thm. 2 sampling) and
    their resolution (intersect_and_resolve). Lets a caller check a result
    whose step-7 picks came from elsewhere."""
    N = x.shape[0]
    t = template_values(t) if t.dtype.kind == "f" else t
    cs = candidate_set_thm2 if thm2 else candidate_set
    return intersect_and_resolve(x, t, [cs(int(m), int(M), N) for m, M in zip(picks, moduli)])


def ftm(x: np.ndarray, t: np.ndarray, M1: int, M2: int, corr: str = "direct") -> Dict:
    """Algorithm 1 steps 3-9 for decoded x (int64/float64) and template t.

    Returns every intermediate: folds y1, y2 (length M+K-1), correlations
    r1, r2 (length M), the step-7 maxima m1, m2, the candidate sets, their
    intersection I and the recovered shift with its status (R6)."""
    N = x.shape[0]
    t = template_values(t) if t.dtype.kind == "f" else t
    K = t.shape[0]
    y1 = fold(x, M1, K)                                        # step 3
    y2 = fold(x, M2, K)
    if corr == "direct":                                      # steps 4-6
        r1, r2 = correlate(y1, t, M1), correlate(y2, t, M2)
    else:
        r1, r2 = correlate_fft(y1, t, M1), correlate_fft(y2, t, M2)
        if x.dtype.kind == "i" and t.dtype.kind == "i":
            # integer correlations: the float64 FFT error is far below 1/2
            r1, r2 = np.rint(r1).astype(np.int64), np.rint(r2).astype(np.int64)
    m1, m2 = argmax_first(r1), argmax_first(r2)               # step 7
    S1, S2 = candidate_set(m1, M1, N), candidate_set(m2, M2, N)  # step 8
    res = intersect_and_resolve(x, t, [S1, S2])               # step 9
    return dict(M1=M1, M2=M2, y1=y1, y2=y2, r1=r1, r2=r2, m1=m1, m2=m2, S1=S1, S2=S2, **res)


# ---------------------------------------------------------------------------
# The second sampling matrix of Thm. 2: Phi = [Phi_M ... Phi_M] with Phi_M = I_M
# acting on x zero-padded to a multiple of M (the paper pads when M does not
# divide N). The fold has length M and the correlation with the template is
# circular with period M: T^ = circ([t 0]) of size M x M (reading R13).
# ---------------------------------------------------------------------------

def fold_thm2(x: np.ndarray, M: int) -> np.ndarray:
    """y = Phi x' (Thm. 2): y_k = sum_l x'_{k + l M}, k < M, x' = x padded with zeros to L M."""
    N = x.shape[0]
    L = ceil_div(N, M)
    xp = np.zeros(L * M, dtype=x.dtype)
    xp[:N] = x
    return xp.reshape(L, M).sum(axis=0)


def correlate_circular(y: np.ndarray, t: np.ndarray, M: int) -> np.ndarray:
    """(T^ y)_j = sum_{i<K} t_i y_{(j+i) mod M}, j < M, T^ = circ([t 0_{M-K}])."""
    K = t.shape[0]
    kind = np.int64 if (y.dtype.kind == "i" and t.dtype.kind == "i") else np.float64
    r = np.zeros(M, dtype=kind)
    for i in range(K):
        r += t[i].astype(kind) * np.roll(y, -i).astype(kind)
    return r


def candidate_set_thm2(m_tilde: int, M: int, N: int) -> Set[int]:
    """{m~ + l M : l < ceil(N/M)} inside the signal (positions in the zero
    padding are not shifts of x) (R13)."""
    return {int(m_tilde + i * M) for i in range(ceil_div(N, M)) if m_tilde + i * M < N}


def ftm_thm2(x: np.ndarray, t: np.ndarray, M1: int, M2: int) -> Dict:
    """Algorithm 1 with the Thm. 2 sampling matrix in step 3 (fold of the
    zero-padded signal, length M) and the circular correlation of period M
    in steps 4-6; steps 7-9 as in ftm()."""
    N = x.shape[0]
    t = template_values(t) if t.dtype.kind == "f" else t
    y1, y2 = fold_thm2(x, M1), fold_thm2(x, M2)
    r1, r2 = correlate_circular(y1, t, M1), correlate_circular(y2, t, M2)
    m1, m2 = argmax_first(r1), argmax_first(r2)
    S1, S2 = candidate_set_thm2(m1, M1, N), candidate_set_thm2(m2, M2, N)
    res = intersect_and_resolve(x, t, [S1, S2])
    return dict(M1=M1, M2=M2, y1=y1, y2=y2, r1=r1, r2=r2, m1=m1, m2=m2, S1=S1, S2=S2, **res)


# ---------------------------------------------------------------------------
# Steps 2-9 with alpha > 2 pairwise co-prime moduli (Thm. 4: a residue
# system whose product reaches N determines the shift uniquely), reading R14
# for their choice.
# ---------------------------------------------------------------------------

def least_s3(N: int) -> int:
    """Least integer s with s (s+1) (s+2) > N."""
    s = max(1, int(round(N ** (1.0 / 3.0))) - 2)
    while s * (s + 1) * (s + 2) <= N:
        s += 1
    while s > 1 and (s - 1) * s * (s + 1) > N:
        s -= 1
    return s


def plan3(N: int, K: int, mode: str = "paper", M1: int = 0, M2: int = 0, M3: int = 0,
          allow_ambig: bool = False) -> Tuple[int, int, int]:
    """Three moduli (R14): "paper" the consecutive integers c, c+1, c+2 from
    the least odd c >= K (pairwise co-prime); "auto" the same from the least
    odd c >= max(K, s), s(s+1)(s+2) > N; "explicit" the caller's."""
    if mode in ("paper", "auto"):
        c = K if mode == "paper" else max(K, least_s3(N))
        c += 1 - c % 2
        M1, M2, M3 = c, c + 1, c + 2
    elif mode != "explicit":
        raise ValueError(mode)
    Ms = (M1, M2, M3)
    if min(Ms) < K:
        raise ValueError("moduli must be >= K")
    for i in range(3):
        for j in range(i + 1, 3):
            if math.gcd(Ms[i], Ms[j]) != 1:
                raise ValueError("moduli must be pairwise co-prime")
    if M1 * M2 * M3 <= N and not allow_ambig:
        raise ValueError("M1*M2*M3 must exceed N")
    return M1, M2, M3


def ftm_multi(x: np.ndarray, t: np.ndarray, moduli, corr: str = "direct") -> Dict:
    """Algorithm 1 with any number of moduli: steps 3-8 for each modulus and
    the intersection of all candidate sets in step 9 (Thm. 4)."""
    N = x.shape[0]
    t = template_values(t) if t.dtype.kind == "f" else t
    K = t.shape[0]
    ys, rs, ms, Ss = [], [], [], []
    for M in moduli:
        y = fold(x, M, K)
        r = correlate(y, t, M) if corr == "direct" else correlate_fft(y, t, M)
        if corr != "direct" and x.dtype.kind == "i" and t.dtype.kind == "i":
            r = np.rint(r).astype(np.int64)
        m = argmax_first(r)
        ys.append(y)
        rs.append(r)
        ms.append(m)
        Ss.append(candidate_set(m, M, N))
    res = intersect_and_resolve(x, t, Ss)
    return dict(moduli=tuple(moduli), ys=ys, rs=rs, ms=ms, Ss=Ss, **res)


def match_query(q, corr: str = "direct") -> Dict:
    """Plan + FTM for a workloads.Query-like object (q.meta["thm2"]: the
    Thm. 2 sampling variant)."""
    x = decode(q.x, q.xdtype, q.N)
    if q.meta.get("three"):
        Ms = plan3(q.N, q.K, q.mode, q.M1, q.M2, q.meta.get("M3", 0), q.allow_ambig)
        return ftm_multi(x, q.t, Ms, corr=corr)
    M1, M2 = plan(q.N, q.K, q.mode, q.M1, q.M2, q.allow_ambig)
    if q.meta.get("thm2"):
        return ftm_thm2(x, q.t, M1, M2)
    return ftm(x, q.t, M1, M2, corr=corr)


# ---------------------------------------------------------------------------
# Full search: the plain definition m = argmax_k (Tx)_k (Eq. 1, Sec. 3).
# ---------------------------------------------------------------------------

def full_search_values(x: np.ndarray, t: np.ndarray) -> np.ndarray:
    """(Tx)_k for every k in [0, N), computed directly in O(NK)."""
    N = x.shape[0]
    K = t.shape[0]
    t = template_values(t) if t.dtype.kind == "f" else t
    acc = np.zeros(N, dtype=np.int64 if (x.dtype.kind == "i" and t.dtype.kind == "i") else np.float64)
    for i in range(K):
        acc += t[i] * np.roll(x, -i)
    return acc


def full_search_fft(x: np.ndarray, t: np.ndarray) -> np.ndarray:
    """(Tx)_k for every k by one length-N FFT correlation in float64; for
    integer inputs the values are rounded to the nearest integer."""
    N = x.shape[0]
    K = t.shape[0]
    tp = np.zeros(N)
    tp[:K] = t
    v = np.fft.irfft(np.conj(np.fft.rfft(tp)) * np.fft.rfft(x.astype(np.float64)), n=N)
    if x.dtype.kind == "i" and np.all(np.asarray(t) == np.round(t)):
        return np.rint(v).astype(np.int64)
    return v


def full_search(x: np.ndarray, t: np.ndarray) -> int:
    N, K = x.shape[0], t.shape[0]
    v = full_search_values(x, t) if N * K <= (1 << 22) else full_search_fft(x, t)
    return argmax_first(v)


# ---------------------------------------------------------------------------
# Matrices of Sec. 2-3, written out for tiny sizes (used by the theorem pins).
# ---------------------------------------------------------------------------

def circ(v: np.ndarray) -> np.ndarray:
    """circ(v): first row v, every next row the previous one rotated right by
    one (Sec. 2)."""
    n = v.shape[0]
    return np.stack([np.roll(v, j) for j in range(n)])


def phi_matrix(N: int, M: int, rows: int) -> np.ndarray:
    """D_rows(circ(r)) with r_k = 1 iff k mod M = 0, 0 <= k < N (Eq. (3))."""
    r = np.array([1 if k % M == 0 else 0 for k in range(N)], dtype=np.int64)
    return circ(r)[:rows]


def T_matrix(t: np.ndarray, N: int) -> np.ndarray:
    """T = circ([t 0_{N-K}]) (Sec. 3)."""
    K = t.shape[0]
    return circ(np.concatenate([t, np.zeros(N - K, dtype=t.dtype)]))


def thm5_fold_failure_bound(N: int, K: int, M: int) -> float:
    """Per-modulus failure bound of Thm. 5: M e^{-K/(8 ceil(N/M))} + 4(ceil(N/M)-1)/K."""
    L = ceil_div(N, M)
    return M * math.exp(-K / (8.0 * L)) + 4.0 * (L - 1) / K


def thm3_condition(tx: np.ndarray, m: int, M: int) -> bool:
    """Thm. 3 hypothesis: (Tx)_m / (2 ceil(N/M) + 1) > max_{k != m} (Tx)_k."""
    N = tx.shape[0]
    L = ceil_div(N, M)
    others = np.delete(tx, m)
    return tx[m] / (2 * L + 1) > others.max()
