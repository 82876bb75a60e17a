"""Seeded synthetic inputs for NNCP workloads (shared by the tests, bench and smoke).

This module only draws random numbers and assembles tensors from them; it holds
none of the decomposition's arithmetic (no MTTKRP, no NLS update, no fit).
Every tensor is returned as a flat float32 numpy vector stored mode-1-fastest
(linear index i_1 + I_1*(i_2 + I_2*(...))), together with its dims; factor
matrices are float32 I_n x R arrays, row-major (R contiguous per row).

Generator recipe (numpy PCG64 via ``np.random.default_rng(seed)``, ``random()``
is U[0,1) in float64):
  * low-rank + additive noise: draw the N true factors as ``random((I_n, R))``
    in mode order, then the noise as ``noise * random(I)`` in linear order; the
    exact model is formed in float64 and the sum rounded to nearest float32.
    The paper's own synthetic data are exact low rank without noise (Sec. V-A);
    ``noise=0`` reproduces that.
  * initial factors: ``random((I_n, R))`` in mode order from a second seed.
"""

from __future__ import annotations

import math

import numpy as np

__all__ = [
    "model_tensor",
    "lowrank_plus_noise",
    "init_factors",
    "hsi_timelapse",
    "batch_problem",
    "serving_request",
    "poisson_arrivals",
]


def model_tensor(factors, dims):
    """Dense float64 sum of the rank-one outer products of ``factors`` (mode-1 fastest)."""
    dims = tuple(int(d) for d in dims)
    N = len(dims)
    R = factors[0].shape[1]
    # rows indexed by (i_N, ..., i_2) with i_2 fastest, built by repeated row-wise
    # products; then one matrix product against the mode-1 factor
    P = np.asarray(factors[N - 1], dtype=np.float64)
    for m in range(N - 2, 0, -1):
        F = np.asarray(factors[m], dtype=np.float64)
        P = (P[:, None, :] * F[None, :, :]).reshape(-1, R)
    A1 = np.asarray(factors[0], dtype=np.float64)
    if N == 1:
        return A1.sum(axis=1)
    return (P @ A1.T).reshape(-1)


def lowrank_plus_noise(dims, R, seed, noise=0.01):
    """Nonnegative rank-R U[0,1) model plus i.i.d. U[0, noise) additive noise."""
    dims = tuple(int(d) for d in dims)
    rng = np.random.default_rng(seed)
    factors = [rng.random((d, R)) for d in dims]
    x = model_tensor(factors, dims)
    if noise:
        x += noise * rng.random(x.size)
    return x.astype(np.float32), [f.astype(np.float32) for f in factors]


def init_factors(dims, R, seed):
    """Initial factors, U[0,1), drawn in mode order."""
    rng = np.random.default_rng(seed)
    return [rng.random((int(d), R)).astype(np.float32) for d in dims]


def _gauss_smooth(col, sigma, radius):
    """1-D Gaussian filter with mirror (reflect) boundary."""
    t = np.arange(-radius, radius + 1, dtype=np.float64)
    k = np.exp(-0.5 * (t / sigma) ** 2)
    k /= k.sum()
    padded = np.pad(col, radius, mode="reflect")
    return np.convolve(padded, k, mode="valid")


def hsi_timelapse(dims=(512, 512, 32, 16), R=24, seed=0, sigma=8.0, radius=32,
                  mult_noise=0.02):
    """4-way spatial x spatial x band x time tensor shaped like time-lapse HSI.

    Spatial factor columns: U[0,1) fields smoothed by a Gaussian (sigma px,
    given radius, mirror boundary).  Band factor columns: sums of 3 Gaussian
    peaks, centre ~ U[0, I_3), width ~ U[1, 4), amplitude ~ U[0.5, 1.5).  Time
    factor columns: U[0.5, 1.5).  Noise: X * (1 + mult_noise * v), v ~ U[-1, 1).
    Draw order: spatial 1, spatial 2, peak centres, widths, amplitudes, time,
    noise.
    """
    dims = tuple(int(d) for d in dims)
    I1, I2, I3, I4 = dims
    rng = np.random.default_rng(seed)
    s1 = rng.random((I1, R))
    s2 = rng.random((I2, R))
    s1 = np.stack([_gauss_smooth(s1[:, r], sigma, radius) for r in range(R)], axis=1)
    s2 = np.stack([_gauss_smooth(s2[:, r], sigma, radius) for r in range(R)], axis=1)
    mu = rng.random((R, 3)) * I3
    w = 1.0 + 3.0 * rng.random((R, 3))
    a = 0.5 + rng.random((R, 3))
    b = np.arange(I3, dtype=np.float64)[:, None]
    band = np.zeros((I3, R))
    for p in range(3):
        band += a[:, p] * np.exp(-((b - mu[:, p]) ** 2) / (2.0 * w[:, p] ** 2))
    time = 0.5 + rng.random((I4, R))
    factors = [s1, s2, band, time]
    x = model_tensor(factors, dims)
    x *= 1.0 + mult_noise * (2.0 * rng.random(x.size) - 1.0)
    return x.astype(np.float32), [f.astype(np.float32) for f in factors]


def batch_problem(t, lo=16, hi=128, ranks=(4, 8, 16), noise=0.01):
    """Tensor t of the batched workload: 3-way, I_n log-uniform in [lo, hi].

    Seeds: 10000 + t for the tensor, 20000 + t for the initial factors.
    Draw order: 3 mode lengths, rank index, factors, noise.
    """
    rng = np.random.default_rng(10000 + t)
    dims = tuple(int(round(math.exp(v))) for v in
                 rng.uniform(math.log(lo), math.log(hi), size=3))
    R = int(ranks[int(rng.integers(len(ranks)))])
    factors = [rng.random((d, R)) for d in dims]
    x = model_tensor(factors, dims)
    x += noise * rng.random(x.size)
    H0 = init_factors(dims, R, 20000 + t)
    return dims, R, x.astype(np.float32), H0


def serving_request(q, lo=16, hi=256, max_elems=64 << 20, ranks=(8, 16, 32, 64),
                    noise_frac=0.02):
    """Request q of the serving workload.

    Order uniform in {3, 4, 5}; mode lengths log-uniform in [lo, hi], the
    whole shape redrawn while the element count exceeds ``max_elems``; R from
    ``ranks``; true rank uniform in [ceil(R/2), 2R]; U[0,1) true factors; additive
    U[0, noise_frac * mean(exact)) noise.  Seeds 30000 + q (tensor) and
    40000 + q (initial factors).
    """
    rng = np.random.default_rng(30000 + q)
    N = int(rng.integers(3, 6))
    while True:
        dims = tuple(int(round(math.exp(v))) for v in
                     rng.uniform(math.log(lo), math.log(hi), size=N))
        if int(np.prod(dims, dtype=np.int64)) <= max_elems:
            break
    R = int(ranks[int(rng.integers(len(ranks)))])
    true_rank = int(rng.integers((R + 1) // 2, 2 * R + 1))
    factors = [rng.random((d, true_rank)) for d in dims]
    x = model_tensor(factors, dims)
    x += noise_frac * float(x.mean()) * rng.random(x.size)
    H0 = init_factors(dims, R, 40000 + q)
    return dims, R, x.astype(np.float32), H0


def poisson_arrivals(count, rate_per_s, seed=5):
    """Arrival times (s) of a Poisson stream: cumulative exponential gaps."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
