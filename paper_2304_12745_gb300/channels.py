"""Seeded synthetic inputs: channels H, user targets t and per-layer parameters.

This module holds no part of the precoder's arithmetic.  It only draws random
inputs, and it is the one module that both the GPU path and the FP64 oracle's
tests read their inputs from.  Every draw comes from numpy's counter-based
Philox generator keyed by an explicit seed, so a batch is reproducible on any
machine; for the Rayleigh and log-normal families the first b instances of a batch
are also the batch of b instances with the same seed.

Channel families (all complex64, layout [B][K][M], row k = user k, column m =
antenna m, as in Sec. II-A of the paper):

* ``rayleigh``       i.i.d. CN(0, 1) entries (Sec. VI-A: the paper trains and tests
                     on these).
* ``lognormal``      CN(0, 1) rows scaled by sqrt(beta_k), beta_k = 10^(sigma_dB z_k / 10),
                     z_k ~ N(0, 1) (large-scale fading with sigma_dB = 8 dB on power).
* ``rician_ula``     h_k = sqrt(kappa/(kappa+1)) e^{j phi_k} a(theta_k) + sqrt(1/(kappa+1)) g_k,
                     a_m(theta) = e^{j pi m sin theta} (half-wavelength ULA),
                     kappa_dB ~ U[kd_lo, kd_hi], theta ~ U[-pi/2, pi/2), phi ~ U[0, 2 pi),
                     g_k ~ CN(0, I).

The five workloads of the benchmark suite are in ``WORKLOADS``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def rng(seed: int, stream: int = 0) -> np.random.Generator:
    """Philox generator for (seed, stream): independent streams per purpose."""
    return np.random.Generator(np.random.Philox(key=[seed & 0xFFFFFFFFFFFFFFFF, stream]))


def _cn(g: np.random.Generator, shape) -> np.ndarray:
    """CN(0, 1) samples as complex64 (real and imaginary parts each N(0, 1/2))."""
    x = g.standard_normal((*shape, 2), dtype=np.float32)
    x *= np.float32(math.sqrt(0.5))
    return x.view(np.complex64)[..., 0]


def rayleigh(B: int, K: int, M: int, seed: int) -> np.ndarray:
    return np.ascontiguousarray(_cn(rng(seed, 1), (B, K, M)))


def lognormal(B: int, K: int, M: int, seed: int, sigma_db: float = 8.0) -> np.ndarray:
    H = _cn(rng(seed, 1), (B, K, M))
    z = rng(seed, 2).standard_normal((B, K))
    beta = 10.0 ** (sigma_db * z / 10.0)
    H *= np.sqrt(beta).astype(np.float32)[:, :, None]
    return np.ascontiguousarray(H)


def rician_ula(B: int, K: int, M: int, seed: int, kd_lo: float = 0.0,
               kd_hi: float = 10.0) -> np.ndarray:
    g = rng(seed, 3)
    kappa = 10.0 ** (g.uniform(kd_lo, kd_hi, (B, K)) / 10.0)
    theta = g.uniform(-math.pi / 2, math.pi / 2, (B, K))
    phi = g.uniform(0.0, 2 * math.pi, (B, K))
    m = np.arange(M)
    los = np.exp(1j * (phi[:, :, None] + math.pi * m[None, None, :] * np.sin(theta)[:, :, None]))
    nlos = _cn(rng(seed, 4), (B, K, M)).astype(np.complex128)
    H = np.sqrt(kappa / (kappa + 1.0))[:, :, None] * los + np.sqrt(1.0 / (kappa + 1.0))[:, :, None] * nlos
    return np.ascontiguousarray(H.astype(np.complex64))


def channels(kind: str, B: int, K: int, M: int, seed: int) -> np.ndarray:
    if kind == "rayleigh":
        return rayleigh(B, K, M, seed)
    if kind == "lognormal":
        return lognormal(B, K, M, seed)
    if kind == "rician":
        return rician_ula(B, K, M, seed)
    raise ValueError(f"unknown channel family {kind!r}")


def targets(B: int, K: int, gamma_db: float | None = None, sigma_nu: float = 1.0) -> np.ndarray:
    """User target amplitudes t_k = sigma_nu * sqrt(gamma_k) as float32 [B][K].

    ``gamma_db=None`` gives unit targets (t_k = 1)."""
    val = 1.0 if gamma_db is None else sigma_nu * math.sqrt(10.0 ** (gamma_db / 10.0))
    return np.full((B, K), val, dtype=np.float32)


def uniform_steps(T: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """Per-layer parameters drawn once from U[lo, hi] (float32 [T])."""
    return rng(seed, 5).uniform(lo, hi, T).astype(np.float32)


@dataclass(frozen=True)
class Workload:
    name: str
    B: int
    K: int
    M: int
    T: int
    family: str
    seed: int
    description: str


WORKLOADS = {
    "tiny": Workload("tiny", 128, 4, 32, 20, "rayleigh", 1,
                     "128 x C^{4x32} i.i.d. CN(0,1), unit targets, T=20, mu_t = 0.05"),
    "fixed": Workload("fixed", 65536, 8, 64, 10, "lognormal", 2,
                      "65,536 x C^{8x64} CN(0,1) rows with 8 dB log-normal gains, unit targets, "
                      "T=10, mu_t ~ U[0.01, 0.1] (seed 2)"),
    "train": Workload("train", 8192, 8, 64, 10, "rayleigh", 4,
                      "batches of 8,192 x C^{8x64} i.i.d. CN(0,1), T=10"),
}

# The paper's training / validation / test sets (Sec. VI-A): i.i.d. CN(0,1) channels
# C^{8x64}, 10^5 for training, 5,000 for validation, 5,000 for testing; per-user
# target SINR 10 dB with sigma_nu = 1 (t = sqrt(10)).  name -> (B, seed)
PAPER_SETS = {"train": (100_000, 300), "validation": (5_000, 301), "test": (5_000, 302)}


def paper_set(name: str, chunk: int = 10_000) -> np.ndarray:
    """One of the paper-setting channel sets, complex64 [B][8][64], drawn in chunks
    of `chunk` instances (chunk i uses seed * 1000 + i)."""
    B, seed = PAPER_SETS[name]
    parts = [rayleigh(min(chunk, B - lo), 8, 64, seed=seed * 1000 + i)
             for i, lo in enumerate(range(0, B, chunk))]
    return np.concatenate(parts)


UNEVEN_SHAPES = ((32, 4), (64, 8), (128, 16), (256, 32))  # (M, K) buckets of the uneven workload


def uneven_shapes(B: int, seed: int) -> np.ndarray:
    """(M, K) per instance drawn uniformly from ``UNEVEN_SHAPES`` -> int32 [B][2]."""
    idx = rng(seed, 6).integers(0, len(UNEVEN_SHAPES), B)
    return np.asarray(UNEVEN_SHAPES, dtype=np.int32)[idx]


def uneven_channels(shapes: np.ndarray, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Rician ULA channels for an uneven batch, packed instance after instance.

    Returns (pool, h_off): pool is complex64 holding instance b's K x M channel at
    element offset h_off[b]; each bucket's instances are drawn together with
    ``rician_ula`` (seed + bucket index)."""
    shapes = np.asarray(shapes)
    sizes = shapes[:, 0].astype(np.int64) * shapes[:, 1]
    h_off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    pool = np.empty(int(sizes.sum()), dtype=np.complex64)
    for i, (M, K) in enumerate(UNEVEN_SHAPES):
        idx = np.nonzero((shapes[:, 0] == M) & (shapes[:, 1] == K))[0]
        if len(idx) == 0:
            continue
        Hb = rician_ula(len(idx), K, M, seed + i).reshape(len(idx), K * M)
        pool[h_off[idx][:, None] + np.arange(K * M)[None, :]] = Hb
    return pool, h_off


def fixed_workload_steps(T: int = 10) -> np.ndarray:
    return uniform_steps(T, 0.01, 0.1, seed=2)


def paper_eta(K: int, M: int) -> float:
    """1 / L~ with the Marchenko-Pastur edge L~ = (sqrt K + sqrt M)^2 (Sec. V)."""
    return 1.0 / (math.sqrt(K) + math.sqrt(M)) ** 2
