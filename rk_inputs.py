"""Seeded synthetic inputs for the RK / RKA / RKAB path.

Shared by the oracle tests, the CUDA-path tests and ``bench.py``; it holds
none of the method's arithmetic (no norms, sampling, projections or
averages), only random draws and the construction of the right-hand side.

The shapes and value distributions follow the workloads of the paper
(Section 3.1: dense overdetermined systems, consistent ``b = A x*`` and an
inconsistent variant ``b + xi`` with Gaussian noise) at the sizes of the
benchmark workloads; entries are iid N(0, 1) unless a row-scale spread
is asked for (rows multiplied by ``10**U(-d, d)``).

Each quantity draws from its own stream so that changing one shape does not
change the others: A <- 1, x* <- 2, noise <- 3, row scales <- 4, x_t <- 5.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

STREAM_A, STREAM_XSTAR, STREAM_NOISE, STREAM_ROWSCALE, STREAM_XT = 1, 2, 3, 4, 5


def _rng(seed: int, stream: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(stream)])


@dataclass
class System:
    A: np.ndarray          # (m, n) float32, C-contiguous
    b: np.ndarray          # (m,) float32
    x_star: np.ndarray     # (n,) float32 generator of b
    noise: float           # std of the added noise (0 for a consistent system)


def gaussian_system(m: int, n: int, seed: int = 0, noise: float = 0.0,
                    row_scale_decades: float = 0.0) -> System:
    """A iid N(0,1) (optionally rows scaled by 10**U(-d, d)), x* iid N(0,1),
    b = fl32(A x* + e), the product taken in FP64 from the FP32 values."""
    A = _rng(seed, STREAM_A).standard_normal((m, n), dtype=np.float32)
    if row_scale_decades:
        sc = 10.0 ** _rng(seed, STREAM_ROWSCALE).uniform(-row_scale_decades,
                                                          row_scale_decades, size=m)
        A *= sc.astype(np.float32)[:, None]
    xs = _rng(seed, STREAM_XSTAR).standard_normal(n, dtype=np.float32)
    b64 = A.astype(np.float64) @ xs.astype(np.float64)
    if noise:
        b64 = b64 + noise * _rng(seed, STREAM_NOISE).standard_normal(m)
    return System(A=A, b=b64.astype(np.float32), x_star=xs, noise=float(noise))


def target_vector(n: int, seed: int = 0) -> np.ndarray:
    """x_t ~ N(0,1) for the loss 0.5 ||x - x_t||^2 of the differentiation form."""
    return _rng(seed, STREAM_XT).standard_normal(n, dtype=np.float32)


def gaussian_system_torch(m: int, n: int, seed: int = 0, noise: float = 0.0,
                          row_scale_decades: float = 0.0, device: str = "cuda",
                          lda: int | None = None):
    """Same recipe drawn directly in device memory with torch's generator
    (for sizes too large to draw on the host).  Values differ from
    :func:`gaussian_system`.  Returns (A (m, lda) float32 with the first n
    columns used, b, x_star)."""
    import torch

    lda = n if lda is None else lda

    def gen(stream):
        g = torch.Generator(device=device)
        g.manual_seed(int(seed) * 1000003 + stream)
        return g

    A = torch.empty((m, lda), dtype=torch.float32, device=device)
    if lda > n:
        A[:, n:].zero_()
    A[:, :n].normal_(generator=gen(STREAM_A))
    if row_scale_decades:
        u = torch.empty(m, dtype=torch.float64, device=device).uniform_(
            -row_scale_decades, row_scale_decades, generator=gen(STREAM_ROWSCALE))
        A[:, :n] *= (10.0 ** u).to(torch.float32)[:, None]
    xs = torch.empty(n, dtype=torch.float32, device=device).normal_(generator=gen(STREAM_XSTAR))
    b64 = torch.zeros(m, dtype=torch.float64, device=device)
    chunk = max(1, (1 << 28) // max(n, 1))
    xs64 = xs.to(torch.float64)
    for r0 in range(0, m, chunk):
        r1 = min(m, r0 + chunk)
        b64[r0:r1] = A[r0:r1, :n].to(torch.float64) @ xs64
    if noise:
        b64 += noise * torch.empty(m, dtype=torch.float64, device=device).normal_(
            generator=gen(STREAM_NOISE))
    return A, b64.to(torch.float32), xs
