"""Seeded synthetic inputs for subsampled-circulant template matching.

This module is shared by the CPU oracle, the tests and the benchmark. It
only *generates* inputs: signals, planted templates and noise. It holds none
of the matcher's arithmetic (no folding, no correlation, no recovery).

Every generator takes an explicit integer seed and uses numpy's PCG64, so a
workload is reproducible on any host. The shapes and value distributions
follow the paper's experiments (Section 4): a +-1 code x, a template cut from
x at a uniformly random cyclic shift, optional template bit flips or Gaussian
noise.

Signal storage types (names match the library's tm_dtype):
  "i8"   int8 bytes holding +1 / -1
  "bits" uint8 bytes, bit-packed, least significant bit first; bit 1 means +1
         and bit 0 means -1
  "f16"  IEEE half
  "f32"  IEEE single
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

DTYPES = ("i8", "bits", "f16", "f32")
MODES = ("auto", "paper", "explicit")


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def pm1_signal(rng: np.random.Generator, N: int) -> np.ndarray:
    """iid uniform +-1 code of length N, stored as int8."""
    b = rng.integers(0, 2, size=int(N), dtype=np.int8)
    b *= 2
    b -= 1
    return b


def gaussian_signal(rng: np.random.Generator, N: int, dtype=np.float32) -> np.ndarray:
    return rng.standard_normal(int(N), dtype=np.float32).astype(dtype, copy=False)


def cyclic_window(x: np.ndarray, k: int, K: int) -> np.ndarray:
    """x[(k + i) mod N] for i < K, as float32 (the planted template)."""
    N = x.shape[0]
    idx = (np.arange(K, dtype=np.int64) + int(k)) % N
    return x[idx].astype(np.float32)


def flip_entries(rng: np.random.Generator, t: np.ndarray, p: float) -> np.ndarray:
    """Negate each entry independently with probability p."""
    if p <= 0.0:
        return t
    mask = rng.random(t.shape[0]) < p
    out = t.copy()
    out[mask] = -out[mask]
    return out


def add_gaussian(rng: np.random.Generator, v: np.ndarray, sigma: float) -> np.ndarray:
    if sigma <= 0.0:
        return v
    return (v.astype(np.float64) + sigma * rng.standard_normal(v.shape[0])).astype(v.dtype)


def pack_bits(x_pm1: np.ndarray) -> np.ndarray:
    """Pack a +-1 code into bytes, LSB first, bit 1 <-> +1.

    The length is padded with zero bits (read as -1) up to a whole byte;
    consumers use N, not the byte count, to know the code length."""
    return np.packbits((x_pm1 > 0).astype(np.uint8), bitorder="little")


@dataclass
class Query:
    """One matching problem: signal x of length N, template t of length K."""
    x: np.ndarray              # storage array (see module doc for the layout)
    xdtype: str                # one of DTYPES
    N: int
    K: int
    t: np.ndarray              # float32[K]
    k_star: int                # planted cyclic shift
    mode: str = "paper"        # one of MODES
    M1: int = 0                # only for mode == "explicit"
    M2: int = 0
    allow_ambig: bool = False  # accept M1*M2 <= N (several CRT solutions)
    seed: int = 0
    meta: dict = field(default_factory=dict)


def planted_query(seed: int, N: int, K: int, xdtype: str = "i8", flip_p: float = 0.0,
                  t_sigma: float = 0.0, mode: str = "paper", allow_ambig: bool = False,
                  M1: int = 0, M2: int = 0) -> Query:
    """A +-1 (or N(0,1) real) signal with a template cut at a random shift.

    The shift k* ~ U[0, N). The template is then optionally corrupted by
    independent sign flips (probability flip_p) and additive N(0, t_sigma^2)
    noise."""
    rng = rng_for(seed)
    if xdtype in ("i8", "bits"):
        x = pm1_signal(rng, N)
    elif xdtype in ("f16", "f32"):
        x = gaussian_signal(rng, N, np.float32)
    else:
        raise ValueError(xdtype)
    k_star = int(rng.integers(0, N))
    t = cyclic_window(x, k_star, K)
    t = flip_entries(rng, t, flip_p)
    t = add_gaussian(rng, t, t_sigma)
    if xdtype == "bits":
        xs = pack_bits(x)
    elif xdtype == "f16":
        xs = x.astype(np.float16)
    else:
        xs = x
    return Query(x=xs, xdtype=xdtype, N=int(N), K=int(K), t=t.astype(np.float32),
                 k_star=k_star, mode=mode, M1=M1, M2=M2, allow_ambig=allow_ambig, seed=seed)


# ---------------------------------------------------------------------------
# Named workloads. Sizes follow the five benchmark configurations:
#   single   : N=65536 +-1 int8, K=1024, noiseless, M1=K, M2=K+1
#   batch64  : 64 queries, N=2^24 +-1 (int8 or bit-packed), K=4096, flips p=0.05
#   sweep    : N=2^22 +-1, K in {256..16384}, flips p=0.1, M1=K, M2=K+1
#   uneven   : N log-uniform in [2^14, 2^24], K log-uniform in [2^8, 2^13],
#              half +-1 int8 / half N(0,1) fp32, template noise N(0, 0.3^2),
#              automatic moduli
# ---------------------------------------------------------------------------

def single_query(seed: int = 1) -> Query:
    return planted_query(seed, 65536, 1024, "i8", mode="paper")


def batch64(seed: int = 100, n: int = 64, N: int = 1 << 24, K: int = 4096,
            xdtype: str = "i8", flip_p: float = 0.05) -> List[Query]:
    return [planted_query(seed + i, N, K, xdtype, flip_p=flip_p, mode="paper") for i in range(n)]


SWEEP_KS = (256, 512, 1024, 2048, 4096, 8192, 16384)


def sweep(seed: int = 1000, K: int = 4096, n: int = 256, N: int = 1 << 22,
          flip_p: float = 0.1, mode: str = "paper") -> List[Query]:
    return [planted_query(seed + i, N, K, "i8", flip_p=flip_p, mode=mode,
                          allow_ambig=(mode == "paper")) for i in range(n)]


def uneven_shapes(seed: int, n: int, logN=(14.0, 24.0), logK=(8.0, 13.0)):
    """(N, K, dtype) triples of the uneven-batch mix; K < N always."""
    rng = rng_for(seed)
    out = []
    for _ in range(n):
        N = int(np.floor(2.0 ** rng.uniform(*logN)))
        K = int(np.floor(2.0 ** rng.uniform(*logK)))
        K = min(K, N - 1)
        dt = "i8" if rng.random() < 0.5 else "f32"
        out.append((N, K, dt))
    return out


def uneven(seed: int = 5000, n: int = 4096, t_sigma: float = 0.3,
           logN=(14.0, 24.0), logK=(8.0, 13.0)) -> List[Query]:
    shapes = uneven_shapes(seed, n, logN, logK)
    return [planted_query(seed * 7919 + i, N, K, dt, t_sigma=t_sigma, mode="auto")
            for i, (N, K, dt) in enumerate(shapes)]


def snr_query(seed: int, N: int, K: int, snr_db: float) -> Query:
    """Section 4 noise experiment: x_e = x + e with e ~ N(0, s^2) and
    s^2 = 10^(-SNR/10) (E[x^2] = 1); the template is the clean window."""
    rng = rng_for(seed)
    x = pm1_signal(rng, N)
    k_star = int(rng.integers(0, N))
    t = cyclic_window(x, k_star, K)
    sigma = float(np.sqrt(10.0 ** (-snr_db / 10.0)))
    xe = (x.astype(np.float32) + (sigma * rng.standard_normal(N)).astype(np.float32))
    return Query(x=xe.astype(np.float32), xdtype="f32", N=N, K=K, t=t, k_star=k_star,
                 mode="paper", seed=seed, meta={"snr_db": snr_db})
