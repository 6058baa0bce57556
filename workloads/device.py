"""Seeded synthetic inputs generated directly in device memory.

For throughput runs whose inputs are too large to draw on the host in
reasonable time (the 4096-query uneven mix holds about 25 GB). The shapes
and value distributions are those of the host generators in this package
(same (N, K, type) triples, +-1 int8 or N(0,1) fp32 signals, templates cut
at a uniformly random cyclic shift plus N(0, sigma^2) noise); the values
come from torch's seeded CUDA generator, so they differ from the host
generators' values. Nothing here computes any part of the matcher.
"""
from __future__ import annotations

from typing import List

import numpy as np

from . import rng_for, uneven_shapes


def _gen(device, seed: int):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    return g


def signal(N: int, xdtype: str, seed: int, device="cuda"):
    """A +-1 int8 (xdtype "i8") or N(0,1) float32/float16 signal of length N."""
    import torch
    g = _gen(device, seed)
    if xdtype == "i8":
        x = torch.randint(0, 2, (N,), generator=g, device=device, dtype=torch.int8)
        return x.mul_(2).sub_(1)
    x = torch.randn(N, generator=g, device=device, dtype=torch.float32)
    return x.half() if xdtype == "f16" else x


def template(x, K: int, k_star: int, sigma: float, seed: int):
    """x[(k_star + i) mod N] for i < K (as float32) plus N(0, sigma^2) noise."""
    import torch
    N = x.shape[0]
    idx = (torch.arange(K, device=x.device, dtype=torch.int64) + int(k_star)) % N
    t = x[idx].float()
    if sigma > 0:
        t += sigma * torch.randn(K, generator=_gen(x.device, seed), device=x.device, dtype=torch.float32)
    return t


def uneven(seed: int = 5000, n: int = 4096, t_sigma: float = 0.3, logN=(14.0, 24.0), logK=(8.0, 13.0),
           device="cuda") -> List[dict]:
    """The uneven mix of uneven_shapes(seed, n, ...) in device memory: a list
    of dicts x, t (CUDA tensors), N, K, xdtype, k_star."""
    shapes = uneven_shapes(seed, n, logN, logK)
    rng = rng_for(seed + 1)
    out = []
    for i, (N, K, dt) in enumerate(shapes):
        x = signal(N, dt, seed * 7919 + i, device)
        k_star = int(rng.integers(0, N))
        t = template(x, K, k_star, t_sigma, seed * 7919 + i + (1 << 40))
        out.append(dict(x=x, t=t, N=N, K=K, xdtype=dt, k_star=k_star))
    return out


def pm1_with_noise(N: int, snr_db: float, seed: int, device="cuda"):
    """A +-1 int8 signal x and x_e = x + e, e ~ N(0, sigma^2) iid with
    sigma^2 = 10^(-snr_db/10) (E[x^2] = 1, so the SNR is 1/sigma^2), as
    float32. Returns (x, x_e)."""
    import torch
    x = signal(N, "i8", seed, device)
    sigma = 10.0 ** (-float(snr_db) / 20.0)
    xe = torch.randn(N, generator=_gen(device, seed + (1 << 41)), device=device, dtype=torch.float32)
    xe.mul_(sigma).add_(x)
    return x, xe
