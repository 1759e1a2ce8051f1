"""Seeded synthetic inputs shared by the CUDA path, the oracle tests and the benchmark.

This module draws problem parameters and data only; it holds none of the multigrid
method's arithmetic (no stencils, transfers, smoothers or losses).  Every array it
returns is float32-valued, so both the CUDA library and the FP64 oracle consume
exactly the same numbers.

Workload shapes follow the paper's test problems (Sec. 6): rotated anisotropic
diffusion with angle theta and conductivity ratio eps (Sec. 6.1), variable
coefficients (Sec. 6.2), right-hand sides drawn at random (Sec. 6.1, evaluation
metrics) and random vectors for the training loss (Thm. sbound).
"""
from __future__ import annotations

import math

import numpy as np

SEED_RHS = 1000
SEED_PARAMS = 2000
SEED_GRF = 3000
SEED_TRAIN = 1_000_000


def rotated_params(seed: int, count: int, eps_lo: float = 1e-3, eps_hi: float = 1.0,
                   theta_lo: float = 0.0, theta_hi: float = math.pi) -> list[tuple[float, float]]:
    """(eps, theta) pairs: eps log-uniform in [eps_lo, eps_hi], theta uniform."""
    rng = np.random.default_rng(seed)
    le = rng.uniform(math.log10(eps_lo), math.log10(eps_hi), size=count)
    th = rng.uniform(theta_lo, theta_hi, size=count)
    return [(float(10.0 ** a), float(t)) for a, t in zip(le, th)]


def rhs_uniform(seed: int, n: int) -> np.ndarray:
    """Right-hand side with i.i.d. uniform[-1, 1] entries, float32 [n, n]."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=(n, n)).astype(np.float32)


def gaussian_vectors(seed: int, count: int, n: int) -> np.ndarray:
    """count standard normal vectors on an n x n grid, float32 [count, n, n]."""
    rng = np.random.default_rng(seed)
    return rng.standard_normal(size=(count, n, n), dtype=np.float64).astype(np.float32)


def grf_cells(seed: int, n: int, corr_len: float = 1.0 / 16.0) -> np.ndarray:
    """Cell coefficients a = exp(g) on the (n+1) x (n+1) cells of the unit square.

    g is a stationary Gaussian random field with unit variance and squared-exponential
    covariance exp(-r^2 / (2 corr_len^2)), sampled on the periodic cell-centre lattice
    by circulant embedding: g = IFFT(sqrt(FFT(c)) * FFT(w)) with w white noise.
    Returns float32 [(n+1), (n+1)].
    """
    m = n + 1
    rng = np.random.default_rng(seed)
    k = np.arange(m)
    d = np.minimum(k, m - k) / m
    r2 = d[:, None] ** 2 + d[None, :] ** 2
    cov = np.exp(-r2 / (2.0 * corr_len ** 2))
    lam = np.maximum(np.fft.fft2(cov).real, 0.0)
    w = rng.standard_normal((m, m))
    g = np.fft.ifft2(np.sqrt(lam) * np.fft.fft2(w)).real
    return np.exp(g).astype(np.float32)


def sine_cells(n: int, kappa: float) -> np.ndarray:
    """Cell coefficients a = sin(kappa pi x y) + 1.1 of the variable-coefficient problem of
    Sec. 6.3, evaluated at the centres of the (n+1) x (n+1) cells of the unit square (row =
    y, column = x).  Returns float32 [(n+1), (n+1)]."""
    m = n + 1
    c = (np.arange(m) + 0.5) / m
    return (np.sin(kappa * math.pi * c[:, None] * c[None, :]) + 1.1).astype(np.float32)


def grid_sizes_loguniform(seed: int, count: int, lo: int = 63, hi: int = 2047) -> list[int]:
    """Square interior sizes drawn log-uniform in [lo, hi], snapped to 2^m - 1."""
    rng = np.random.default_rng(seed)
    raw = np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))
    return [int(2 ** round(math.log2(v + 1)) - 1) for v in raw]
