"""Seeded synthetic inputs for singular value soft-thresholding (SVT).

This module is shared by the FP64 oracle, the tests and the benchmark. It holds
input recipes only: no step of the SVT method lives here. Every generator draws
from ``numpy.random.default_rng(seed)`` in FP64 and returns FP32 arrays unless
stated otherwise, so the same seed gives the same bytes on x86 and Arm hosts.

The paper measures on iid Gaussian matrices (Section 3: a 301x300 Gaussian
accuracy test for Fig. 1 and m x (m+1) Gaussian matrices for Fig. 2). The
recipes below keep that structure and add the spectra the evaluation needs:

* ``spectrum_matrix``: ``Q1 diag(sigma) Q2^T`` with Haar-like Q from the QR of a
  Gaussian matrix, for a prescribed spectrum (the 64x64 case with a gap around
  tau = 0.3).
* ``marchenko_pastur``: entries N(0, 1/n); the spectrum fills [0, 2] with no gap.
* ``low_rank_plus_noise``: rank-r signal with singular values uniform in a range,
  plus 0.01 N(0,1) noise.
* ``batch_recipe``: an uneven batch of low-rank-plus-noise matrices with a tau per
  matrix just above the noise edge.
* ``poisson_requests``: a Poisson arrival stream of such requests.
* ``completion_problem``: a low-rank target with a Bernoulli observation mask.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Fixed seeds per workload family (a replicate index is added to them).
SEED_SPECTRUM_64 = 1001
SEED_MP = 1002
SEED_LOWRANK = 1003
SEED_BATCH = 1004
SEED_SERVE = 1005


def _haar(rng: np.random.Generator, n: int, k: int | None = None) -> np.ndarray:
    """n x k matrix with orthonormal columns: QR of a Gaussian, signs fixed by R's diagonal."""
    k = n if k is None else k
    g = rng.standard_normal((n, k))
    q, r = np.linalg.qr(g)
    return q * np.sign(np.diag(r))[None, :]


def spectrum_64_sigma() -> np.ndarray:
    """The 64-value spectrum of the small case: 49 log-spaced values in [1e-2, 0.24]
    and 15 log-spaced values in [0.36, 1]. No value lies in [0.25, 0.35], so every
    singular value is at least 0.06 (6 % of sigma_max = 1) away from tau = 0.3."""
    lo = np.logspace(math.log10(1e-2), math.log10(0.24), 49)
    hi = np.logspace(math.log10(0.36), math.log10(1.0), 15)
    return np.sort(np.concatenate([lo, hi]))[::-1].copy()


def spectrum_matrix(sigma: np.ndarray, m: int, n: int, seed: int) -> np.ndarray:
    """m x n FP32 matrix Q1 diag(sigma) Q2^T with the given singular values
    (len(sigma) = min(m, n)); Q1, Q2 from seeded QR."""
    rng = np.random.default_rng(seed)
    k = min(m, n)
    assert len(sigma) == k
    q1 = _haar(rng, m, k)
    q2 = _haar(rng, n, k)
    return ((q1 * np.asarray(sigma, np.float64)[None, :]) @ q2.T).astype(np.float32)


def spectrum_64(seed: int = SEED_SPECTRUM_64) -> np.ndarray:
    """The 64x64 case with a 6 % gap around tau = 0.3."""
    return spectrum_matrix(spectrum_64_sigma(), 64, 64, seed)


def marchenko_pastur(m: int, n: int | None = None, seed: int = SEED_MP) -> np.ndarray:
    """m x n FP32 matrix with iid N(0, 1/max(m,n)) entries (Marchenko-Pastur spectrum)."""
    n = m if n is None else n
    rng = np.random.default_rng(seed)
    scale = 1.0 / math.sqrt(max(m, n))
    return (rng.standard_normal((m, n)) * scale).astype(np.float32)


def quarter_circle_sigma(n: int) -> np.ndarray:
    """Singular values of an n x n N(0, 1/n) matrix follow the quarter-circle law on
    [0, 2] (density sqrt(4 - s^2) / pi, the square case of Marchenko-Pastur); returns
    its (i - 1/2) / n quantiles, largest first, by bisection on the closed-form
    distribution function. With Haar singular vectors this gives a matrix shaped like
    the benchmark's whose SVD, and hence A_tau, is known exactly."""
    cdf = lambda s: (s * np.sqrt(4.0 - s * s) / 2.0 + 2.0 * np.arcsin(s / 2.0)) / np.pi
    p = (np.arange(n) + 0.5) / n
    lo, hi = np.zeros(n), np.full(n, 2.0)
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        below = cdf(mid) < p
        lo = np.where(below, mid, lo)
        hi = np.where(below, hi, mid)
    return np.ascontiguousarray(np.sort(0.5 * (lo + hi))[::-1])


def mp_noise_sigma(m: int, n: int, scale: float, count: int) -> np.ndarray:
    """Singular values of an m x n matrix of N(0, scale^2) entries follow the
    Marchenko-Pastur law: with y = min/max of the sides and N = the larger side,
    sigma = scale * sqrt(N * lambda), lambda on [(1 - sqrt y)^2, (1 + sqrt y)^2] with
    density sqrt((b - lambda)(lambda - a)) / (2 pi y lambda). Returns `count` of its
    (i - 1/2) / count quantiles, largest first, from the distribution function
    integrated numerically (lambda = a + (b - a)(1 - cos t) / 2 removes the square-root
    endpoints; the square case's 1 / sqrt(lambda) edge becomes a finite limit)."""
    y = min(m, n) / max(m, n)
    a, b = (1.0 - math.sqrt(y)) ** 2, (1.0 + math.sqrt(y)) ** 2
    t = np.linspace(0.0, math.pi, 200001)
    lam = a + (b - a) * (1.0 - np.cos(t)) / 2.0
    with np.errstate(divide="ignore", invalid="ignore"):
        f = ((b - a) / 2.0) ** 2 * np.sin(t) ** 2 / (2.0 * math.pi * y * lam)
    # square case (a = 0): the integrand tends to b / (2 pi y) at lambda = 0
    f = np.where(lam > 0.0, f, b / (2.0 * math.pi * y))
    cdf = np.concatenate([[0.0], np.cumsum(0.5 * (f[1:] + f[:-1]) * np.diff(t))])
    cdf /= cdf[-1]
    p = (np.arange(count) + 0.5) / count
    lam_q = np.interp(p, cdf, lam)
    return np.ascontiguousarray(np.sort(scale * np.sqrt(max(m, n) * lam_q))[::-1])


def low_rank_plus_noise_spectrum(m: int, n: int, rank: int, seed: int, sig_lo: float = 1.0,
                                 sig_hi: float = 10.0, noise: float = 0.01) -> np.ndarray:
    """The singular values of ``low_rank_plus_noise``'s recipe for a known-SVD stand-in:
    `rank` signal values uniform in [sig_lo, sig_hi] and the Marchenko-Pastur quantiles
    of the N(0, noise^2) part for the rest, largest first."""
    rng = np.random.default_rng(seed)
    k = min(m, n)
    sig = np.concatenate([rng.uniform(sig_lo, sig_hi, rank), mp_noise_sigma(m, n, noise, k - rank)])
    return np.ascontiguousarray(np.sort(sig)[::-1])


def low_rank_plus_noise(m: int, n: int, rank: int, seed: int,
                        sig_lo: float = 1.0, sig_hi: float = 10.0,
                        noise: float = 0.01) -> np.ndarray:
    """m x n FP32 matrix U_s diag(sigma_s) V_s^T + noise * N(0,1), sigma_s ~ U[sig_lo, sig_hi]."""
    rng = np.random.default_rng(seed)
    us = _haar(rng, m, rank)
    vs = _haar(rng, n, rank)
    sig = rng.uniform(sig_lo, sig_hi, rank)
    a = (us * sig[None, :]) @ vs.T + noise * rng.standard_normal((m, n))
    return a.astype(np.float32)


def noise_edge(m: int, n: int, noise: float = 0.01) -> float:
    """Upper edge of the noise bulk of an m x n matrix of iid noise * N(0,1) entries."""
    return noise * (math.sqrt(m) + math.sqrt(n))


@dataclass
class BatchItem:
    m: int
    n: int
    rank: int
    tau: float
    seed: int

    def matrix(self) -> np.ndarray:
        return low_rank_plus_noise(self.m, self.n, self.rank, self.seed, 2.0, 10.0)


def batch_recipe(count: int = 256, s_lo: int = 128, s_hi: int = 1024,
                 seed: int = SEED_BATCH) -> list[BatchItem]:
    """Uneven batch: size s log-uniform in [s_lo, s_hi], aspect in {1, 2, 1/2}
    (shapes s x s, s x s/2, s/2 x s), rank uniform in 5..50, signal singular
    values uniform in [2, 10], noise 0.01 N(0,1), and
    tau = noise edge + 0.05 * sigma_max(signal upper bound 10)."""
    rng = np.random.default_rng(seed)
    items = []
    for i in range(count):
        s = int(round(math.exp(rng.uniform(math.log(s_lo), math.log(s_hi)))))
        aspect = int(rng.integers(0, 3))
        if aspect == 0:
            m, n = s, s
        elif aspect == 1:
            m, n = s, max(1, s // 2)
        else:
            m, n = max(1, s // 2), s
        rank = int(rng.integers(5, 51))
        rank = min(rank, m, n)
        tau = noise_edge(m, n) + 0.05 * 10.0
        items.append(BatchItem(m, n, rank, tau, seed * 1000 + i))
    return items


@dataclass
class Request:
    arrival_s: float
    m: int
    n: int
    rank: int
    tau: float
    tier: str  # "bf16" or "fp32"
    seed: int

    def matrix(self) -> np.ndarray:
        return low_rank_plus_noise(self.m, self.n, self.rank, self.seed, 2.0, 10.0)


def poisson_requests(count: int, rate_per_s: float, s_lo: int = 256, s_hi: int = 8192,
                     fp32_fraction: float = 0.3, seed: int = SEED_SERVE) -> list[Request]:
    """Poisson arrival stream: exponential gaps at the given rate, sizes
    log-uniform in [s_lo, s_hi] with aspect as in ``batch_recipe``, tier FP32
    with probability ``fp32_fraction`` else BF16."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate_per_s))
        s = int(round(math.exp(rng.uniform(math.log(s_lo), math.log(s_hi)))))
        aspect = int(rng.integers(0, 3))
        m, n = (s, s) if aspect == 0 else ((s, s // 2) if aspect == 1 else (s // 2, s))
        rank = min(int(rng.integers(5, 51)), m, n)
        tier = "fp32" if rng.uniform() < fp32_fraction else "bf16"
        tau = noise_edge(m, n) + 0.5
        out.append(Request(t, m, n, rank, tau, tier, seed * 100000 + i))
    return out


def completion_problem(n: int = 4096, rank: int = 20, frac: float = 0.2,
                       target_norm: float = 10.0, seed: int = SEED_SERVE + 7):
    """Matrix completion instance: M = L R^T (L, R ~ N(0,1)^{n x rank}) scaled so
    that ||M||_2 is about ``target_norm``, and a Bernoulli(frac) mask Omega.
    Returns (M, mask) as FP32 arrays."""
    rng = np.random.default_rng(seed)
    lft = rng.standard_normal((n, rank))
    rgt = rng.standard_normal((n, rank))
    # ||L R^T||_2 from the 'rank x rank' core of the two thin QR factorisations.
    core = np.linalg.qr(lft)[1] @ np.linalg.qr(rgt)[1].T
    mat = (lft @ rgt.T) * (target_norm / np.linalg.norm(core, 2))
    mask = (rng.uniform(size=(n, n)) < frac)
    return mat.astype(np.float32), mask.astype(np.float32)
