"""Seeded synthetic multi-series inputs and range-query lists.

This module is shared by the CUDA path's tests/bench and by the FP64 oracle's
tests.  It holds no arithmetic of the range-SVD method itself: it only draws
numbers.  The paper's datasets (Activity 382,000x41, Gas 4,107,000x16,
London 350,000x10; Table 2) are not available, so these generators stand in
for them with the same structure: a few smooth latent factors (sinusoids)
mixed into many correlated sensor columns plus white noise (Section 5.1).

Recipe (all draws from numpy ``Generator(PCG64)``):
  * latent signals  s_j(t) = sin(2*pi*f_j*t + phi_j),  f_j ~ U[1e-3, 5e-2]
    cycles/row, phi_j ~ U[0, 2*pi), j = 1..s;
  * mixing          L ~ N(0, 1)^{s x n};  A = S L;
  * noise           + N(0, sigma_noise^2) per entry (sigma_noise = 0.05);
  * optional drift  + per-column random walk with N(0, drift^2) steps.
Rows are generated in fixed chunks of ``CHUNK`` rows, each from its own
sub-stream, so any row range can be produced without generating the rest
(drift excepted: its carry needs the increments of earlier chunks).

Range queries (Section 5.2, Fig. 1): length l ~ log-uniform[l_min, l_max],
t_s ~ U{0 .. T-l}, t_e = t_s + l - 1 (0-based, inclusive).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 1805007540
CHUNK = 8192


@dataclasses.dataclass(frozen=True)
class SeriesSpec:
    T: int            # rows (time)
    n: int            # series (columns); the paper's c
    s: int = 6        # latent sinusoids
    noise: float = 0.05
    drift: float = 0.0
    seed: int = SEED_BASE


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    series: SeriesSpec
    b: int
    k: int
    dtype: str                  # "f64" | "f32" | "bf16"  (input storage type)
    nq: int = 0                 # queries in one batch
    lmin: int = 0
    lmax: int = 0
    single_query: tuple | None = None


# The five workloads the method is measured on (shapes follow the paper's
# Section 5: b ~ 1e3, ranges 1e4..3.2e5 rows, few latent factors).  Where the
# workload definition does not fix the number of latent sinusoids s, s is
# k + 8 (a few more factors than the kept rank, like sensor data whose energy
# sits in a handful of components).  Spectra without a gap after k are drawn
# by ``spectral_rows`` below; the tests run the method on both kinds.
WORKLOADS = {
    "plain_f64": Workload(
        "plain_f64", SeriesSpec(20_000, 32, 6, 0.05, 0.0, SEED_BASE + 0),
        b=500, k=8, dtype="f64", single_query=(1_234, 15_678)),
    "compress_f32": Workload(
        "compress_f32", SeriesSpec(1_048_576, 256, 20, 0.05, 1e-3, SEED_BASE + 1),
        b=1_024, k=16, dtype="f32", nq=1_024, lmin=10_000, lmax=320_000),
    "precision_bf16": Workload(
        "precision_bf16", SeriesSpec(1_048_576, 512, 40, 0.05, 0.0, SEED_BASE + 2),
        b=2_048, k=32, dtype="bf16", nq=1_000, lmin=10_000, lmax=320_000),
    "ragged_batch_f32": Workload(
        "ragged_batch_f32", SeriesSpec(4_194_304, 128, 28, 0.05, 0.0, SEED_BASE + 3),
        b=2_000, k=20, dtype="f32", nq=4_096, lmin=10_000, lmax=320_000),
    "serving_f32": Workload(
        "serving_f32", SeriesSpec(8_388_608, 64, 18, 0.05, 0.0, SEED_BASE + 4),
        b=4_096, k=10, dtype="f32", nq=20_000, lmin=1_000, lmax=1_000_000),
}


def _chunk_rng(seed: int, chunk: int, stream: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64([seed, chunk, stream]))


def _latent_params(spec: SeriesSpec):
    g = np.random.Generator(np.random.PCG64([spec.seed, 0xFAC7]))
    f = g.uniform(1e-3, 5e-2, spec.s)
    phi = g.uniform(0.0, 2.0 * math.pi, spec.s)
    L = g.standard_normal((spec.s, spec.n))
    return f, phi, L


def rows(spec: SeriesSpec, r0: int = 0, r1: int | None = None,
         dtype=np.float64) -> np.ndarray:
    """Rows [r0, r1) of the seeded T x n matrix, row-major, as ``dtype``."""
    if r1 is None:
        r1 = spec.T
    if not (0 <= r0 <= r1 <= spec.T):
        raise ValueError("row range out of bounds")
    f, phi, L = _latent_params(spec)
    out = np.empty((r1 - r0, spec.n), dtype=dtype)
    c0, c1 = r0 // CHUNK, (r1 + CHUNK - 1) // CHUNK
    carry = np.zeros(spec.n)
    if spec.drift > 0.0:
        for c in range(0, c0):
            g = _chunk_rng(spec.seed, c, 2)
            carry += g.standard_normal((CHUNK, spec.n)).sum(axis=0) * spec.drift
    for c in range(c0, c1):
        lo, hi = c * CHUNK, min((c + 1) * CHUNK, spec.T)
        t = np.arange(lo, hi, dtype=np.float64)[:, None]
        block = np.sin(2.0 * math.pi * f[None, :] * t + phi[None, :]) @ L
        block += spec.noise * _chunk_rng(spec.seed, c, 1).standard_normal((hi - lo, spec.n))
        if spec.drift > 0.0:
            inc = _chunk_rng(spec.seed, c, 2).standard_normal((CHUNK, spec.n))[: hi - lo]
            walk = np.cumsum(inc, axis=0) * spec.drift + carry[None, :]
            carry = walk[-1].copy() if hi - lo == CHUNK else carry
            block += walk
        a, z = max(lo, r0), min(hi, r1)
        out[a - r0: z - r0] = block[a - lo: z - lo]
    return out


def queries(T: int, nq: int, lmin: int, lmax: int, seed: int):
    """``nq`` inclusive ranges (t_s, t_e) with log-uniform lengths."""
    g = np.random.Generator(np.random.PCG64([seed, 0x9E4]))
    lmax = min(lmax, T)
    lmin = min(lmin, lmax)
    ln = g.uniform(math.log(lmin), math.log(lmax), nq)
    length = np.clip(np.rint(np.exp(ln)).astype(np.int64), 1, T)
    ts = np.floor(g.uniform(0.0, 1.0, nq) * (T - length + 1)).astype(np.int64)
    ts = np.minimum(ts, T - length)
    te = ts + length - 1
    return ts, te


def poisson_arrivals(rate_hz: float, duration_s: float, seed: int) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process, for the serving loop."""
    g = np.random.Generator(np.random.PCG64([seed, 0xA77]))
    n = int(rate_hz * duration_s * 1.2) + 16
    t = np.cumsum(g.exponential(1.0 / rate_hz, n))
    return t[t < duration_s]


def to_bf16_bits(x: np.ndarray) -> np.ndarray:
    """Round-to-nearest-even float32 -> bfloat16, returned as uint16 bits.

    A storage-format conversion of the input (not part of the method): the
    bf16 workload stores its rows in this format and both sides read the same
    bits.
    """
    f = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32)
    rounding = ((f >> 16) & 1) + 0x7FFF
    return ((f + rounding) >> 16).astype(np.uint16)


def bf16_bits_to_f64(bits: np.ndarray) -> np.ndarray:
    return (bits.astype(np.uint32) << 16).view(np.float32).astype(np.float64)


# --------------------------------------------------------------------------
# Rows with a prescribed spectrum (no gap after the kept rank).
#
# Each row is a_t = z_t D Q^T with z_t ~ N(0, I_n), D = diag(d_1..d_n) and Q a
# seeded random orthogonal n x n matrix: a stationary multi-series whose
# covariance Q D^2 Q^T has eigenvalues d_j^2, so every block of b >= n rows
# has singular values close to sqrt(b) d_j, with no gap unless d has one.
# Families of d_j (j = 1..n):
#   "pow0.5"   j^-0.5             slow power decay
#   "pow1"     j^-1               power decay
#   "geo0.97"  0.97^j             geometric decay
#   "flat64"   1 for j <= 64, then 0.05: 64 equal-strength directions (64
#              near-equal signals) over a noise floor
# --------------------------------------------------------------------------
SPECTRA = ("pow0.5", "pow1", "geo0.97", "flat64")


@dataclasses.dataclass(frozen=True)
class SpectralSpec:
    T: int
    n: int
    family: str
    seed: int = SEED_BASE + 100


def spectrum(family: str, n: int) -> np.ndarray:
    j = np.arange(1, n + 1, dtype=np.float64)
    if family == "pow0.5":
        return j ** -0.5
    if family == "pow1":
        return 1.0 / j
    if family == "geo0.97":
        return 0.97 ** j
    if family == "flat64":
        return np.where(j <= 64, 1.0, 0.05)
    if family.startswith("gap"):
        # "gapK": 1/j for the first K directions, then a floor 1e-4 j^-1/2 -
        # a clear gap after K at every row count, so that truncating to rank
        # K after every row (Algorithm 1 as printed) is well conditioned
        K = int(family[3:])
        return np.where(j <= K, 1.0 / j, 1e-4 / np.sqrt(j))
    if family.startswith("drop"):
        # "dropK": the same with a floor 0.1 j^-1/2 - still a gap after K,
        # but each row's truncation drops enough energy that the row-by-row
        # result differs visibly (~1e-5 sigma_1) from the block's truncated SVD
        K = int(family[4:])
        return np.where(j <= K, 1.0 / j, 0.1 / np.sqrt(j))
    raise ValueError(f"unknown spectrum family {family!r}")


def spectral_rows(spec: SpectralSpec, r0: int = 0, r1: int | None = None,
                  dtype=np.float64) -> np.ndarray:
    """Rows [r0, r1) of the seeded T x n matrix with spectrum ``spec.family``."""
    if r1 is None:
        r1 = spec.T
    if not (0 <= r0 <= r1 <= spec.T):
        raise ValueError("row range out of bounds")
    g = np.random.Generator(np.random.PCG64([spec.seed, 0x5BEC]))
    Q, R = np.linalg.qr(g.standard_normal((spec.n, spec.n)))
    Q *= np.sign(np.diag(R))[None, :]
    M = spectrum(spec.family, spec.n)[:, None] * Q.T          # D Q^T
    out = np.empty((r1 - r0, spec.n), dtype=dtype)
    for c in range(r0 // CHUNK, (r1 + CHUNK - 1) // CHUNK):
        lo, hi = c * CHUNK, min((c + 1) * CHUNK, spec.T)
        Z = _chunk_rng(spec.seed, c, 3).standard_normal((hi - lo, spec.n))
        a, z = max(lo, r0), min(hi, r1)
        out[a - r0: z - r0] = Z[a - lo: z - lo] @ M
    return out
