"""Seeded synthetic input sequences (no wavelet-tree arithmetic lives here).

Both the tests (through the oracle) and the library's benchmark draw their
sequences from this module, so the two sides see identical bytes.  Every
value is a pure function of (seed, index):

* the random stream is splitmix64 (Steele, Lea and Flood, 2014): the j-th
  output for a seed is ``mix(seed + (j + 1) * 0x9E3779B97F4A7C15)`` with the
  published 64-bit finaliser ``mix``;
* a uniform code in [0, sigma) is Lemire's multiply-shift of the top 32 bits,
  ``((x >> 32) * sigma) >> 32``;
* a Zipf(alpha) code first draws a rank r in [1, sigma] with probability
  proportional to r^-alpha by inverting the float64 CDF at
  ``u = (x >> 11) * 2^-53``, then maps it through a seeded permutation of
  [0, sigma) (the codes sorted by the stream of ``seed ^ 0xA5``), so frequent
  codes are scattered over the alphabet.

The named workloads mirror the shapes of the paper's data sets (Section 4,
Table 1): DNA-like sequences over 4 codes, text-like sequences over about a
hundred byte codes, word-id sequences over a large alphabet with Zipf-like
frequencies.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22

SEED_BASE = 20161005


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start .. start+count-1 of the splitmix64 stream of ``seed``."""
    with np.errstate(over="ignore"):
        j = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        return _mix(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + j * GOLDEN)


def sym_dtype(sigma: int):
    """Smallest of uint8 / uint16 / uint32 that holds codes below sigma."""
    if sigma <= 1 << 8:
        return np.uint8
    if sigma <= 1 << 16:
        return np.uint16
    return np.uint32


def _parallel_fill(n: int, dtype, fill) -> np.ndarray:
    out = np.empty(n, dtype=dtype)
    starts = list(range(0, n, _CHUNK))
    if len(starts) <= 1:
        for s in starts:
            out[s:s + _CHUNK] = fill(s, min(_CHUNK, n - s))
        return out
    workers = min(len(starts), os.cpu_count() or 1, 32)

    def job(s):
        out[s:s + _CHUNK] = fill(s, min(_CHUNK, n - s))

    with ThreadPoolExecutor(workers) as ex:
        list(ex.map(job, starts))
    return out


def uniform(n: int, sigma: int, seed: int, dtype=None) -> np.ndarray:
    """n i.i.d. uniform codes in [0, sigma)."""
    dtype = dtype or sym_dtype(sigma)
    sig = np.uint64(sigma)

    def fill(s, c):
        with np.errstate(over="ignore"):
            return (((splitmix64(seed, s, c) >> np.uint64(32)) * sig) >> np.uint64(32)).astype(dtype)

    return _parallel_fill(n, dtype, fill)


_PERM_CACHE: dict = {}
_CDF_CACHE: dict = {}


def permutation(sigma: int, seed: int) -> np.ndarray:
    """A seeded permutation of [0, sigma): the codes ordered by the
    splitmix64 stream of seed ^ 0xA5 (stable sort of the stream's values)."""
    key = (sigma, seed)
    if key not in _PERM_CACHE:
        _PERM_CACHE[key] = np.argsort(splitmix64(seed ^ 0xA5, 0, sigma), kind="stable").astype(np.uint32)
    return _PERM_CACHE[key]


def zipf_cdf(sigma: int, alpha: float) -> np.ndarray:
    key = (sigma, alpha)
    if key not in _CDF_CACHE:
        w = np.arange(1, sigma + 1, dtype=np.float64) ** (-alpha)
        cdf = np.cumsum(w)
        _CDF_CACHE[key] = cdf / cdf[-1]
    return _CDF_CACHE[key]


def zipf(n: int, sigma: int, alpha: float, seed: int, dtype=None) -> np.ndarray:
    """n i.i.d. Zipf(alpha) codes over a seeded permutation of [0, sigma)."""
    dtype = dtype or sym_dtype(sigma)
    cdf = zipf_cdf(sigma, alpha)
    perm = permutation(sigma, seed)
    scale = 1.0 / float(1 << 53)

    def fill(s, c):
        u = (splitmix64(seed, s, c) >> np.uint64(11)).astype(np.float64) * scale
        r = np.searchsorted(cdf, u, side="right")
        np.minimum(r, sigma - 1, out=r)
        return perm[r].astype(dtype)

    return _parallel_fill(n, dtype, fill)


# ------------------------------------------------ locality stress inputs
#
# The paper's locality experiment (Section 4, the cont and rand data sets):
# n symbols over sigma codes, each code written n / sigma times.  cont puts
# them in code order (every level of the tree sees long runs of one node);
# rand puts the same multiset at random positions.  Here rand[j] =
# cont[pi(j)] for a seeded bijection pi of [0, n): on k-bit integers (2^k >=
# n) an offset by the seed, then three rounds of an xorshift and a multiply
# by an odd constant mod 2^k (each step invertible), cycle-walked into
# [0, n).  Both a numpy and a torch form are given; they agree bit for bit.

_LOC_MULS = (0x9E3779B1, 0x85EBCA6B, 0xC2B2AE35)


def _loc_bits(n: int) -> int:
    return max(1, (n - 1).bit_length())


def _loc_round(x, k: int, seed: int, xp_and, xp_xor, xp_shr, xp_mul, xp_add):
    m = (1 << k) - 1
    x = xp_and(xp_add(x, seed & m), m)
    for c in _LOC_MULS:
        x = xp_xor(x, xp_shr(x, max(1, k // 2)))
        x = xp_and(xp_mul(x, c), m)
    return xp_xor(x, xp_shr(x, max(1, (k + 1) // 2)))


def locality_positions(j: np.ndarray, n: int, seed: int) -> np.ndarray:
    """pi(j) for positions j of [0, n) (numpy, uint64)."""
    k = _loc_bits(n)
    u = np.uint64
    with np.errstate(over="ignore"):
        f = lambda x: _loc_round(x, k, seed, lambda a, b: a & u(b), lambda a, b: a ^ b, lambda a, b: a >> u(b),
                                 lambda a, b: a * u(b), lambda a, b: a + u(b))
        x = f(j.astype(np.uint64))
        out = x >= u(n)
        while out.any():
            x[out] = f(x[out])
            out = x >= u(n)
    return x


def locality(n: int, sigma: int, kind: str, seed: int, dtype=np.uint32) -> np.ndarray:
    """The cont or rand sequence (numpy): code floor(q * sigma / n) at
    q = j (cont) or q = pi(j) (rand)."""
    s = np.uint64(sigma)

    def fill(st, c):
        j = np.arange(st, st + c, dtype=np.uint64)
        q = j if kind == "cont" else locality_positions(j, n, seed)
        return ((q * s) // np.uint64(n)).astype(dtype)

    return _parallel_fill(n, dtype, fill)


def locality_torch(n: int, sigma: int, kind: str, seed: int, device, dtype=None):
    """The same sequence generated by torch on `device` (int32 codes, or
    `dtype`), for sizes whose host generation would take long."""
    import torch
    k = _loc_bits(n)
    j = torch.arange(n, dtype=torch.int64, device=device)
    if kind == "cont":
        q = j
    else:
        f = lambda x: _loc_round(x, k, seed, lambda a, b: a & b, lambda a, b: a ^ b, lambda a, b: a >> b,
                                 lambda a, b: a * b, lambda a, b: a + b)
        q = f(j)
        del j
        out = q >= n
        while bool(out.any()):
            q = torch.where(out, f(q), q)
            out = q >= n
    codes = torch.div(q * sigma, n, rounding_mode="floor")
    return codes.to(dtype or torch.int32)


LOCALITY_SIZES = tuple(range(4, 15, 2))   # sigma = 2^y, y in {4, 6, ..., 14}


# ----------------------------------------------------------- named workloads

@dataclass(frozen=True)
class Workload:
    """One single-sequence workload: shape, alphabet, distribution and seed."""
    name: str
    n: int
    sigma: int
    dist: str            # "uniform" or "zipf"
    alpha: float
    seed: int
    width: int           # bytes per symbol

    def generate(self, n: int | None = None) -> np.ndarray:
        """The sequence (or its first n symbols when n is given)."""
        m = self.n if n is None else n
        dt = {1: np.uint8, 2: np.uint16, 4: np.uint32}[self.width]
        if self.dist == "uniform":
            return uniform(m, self.sigma, self.seed, dt)
        return zipf(m, self.sigma, self.alpha, self.seed, dt)


WORKLOADS = {
    # small parity case: 2^20 bytes over 256 codes, uniform (8 levels)
    "u8-uniform-2^20-s256": Workload("u8-uniform-2^20-s256", 1 << 20, 256, "uniform", 0.0, SEED_BASE + 1, 1),
    # text-like: 2^30 bytes, 96 codes, Zipf 1.0 (7 levels); stands in for prot / en.6-8.30
    "u8-text-2^30-s96-zipf1.0": Workload("u8-text-2^30-s96-zipf1.0", 1 << 30, 96, "zipf", 1.0, SEED_BASE + 2, 1),
    # DNA-like: 2^30 bytes over 4 codes, uniform (2 levels); stands in for rna.1GB
    "u8-dna-2^30-s4": Workload("u8-dna-2^30-s4", 1 << 30, 4, "uniform", 0.0, SEED_BASE + 20, 1),
    # word ids: 2^29 uint32 over 2^20 codes, Zipf 1.2 (20 levels); stands in for src.2GB / en.14.30
    "u32-words-2^29-s2^20-zipf1.2": Workload("u32-words-2^29-s2^20-zipf1.2", 1 << 29, 1 << 20, "zipf", 1.2, SEED_BASE + 3, 4),
}


def seq_seed(base: int, idx: int) -> int:
    """Per-sequence seed of a batch: base xor (idx * golden gamma) mod 2^64."""
    return (base ^ ((idx * 0x9E3779B97F4A7C15) & 0xFFFFFFFFFFFFFFFF)) & 0xFFFFFFFFFFFFFFFF


@dataclass(frozen=True)
class SeqSpec:
    n: int
    sigma: int
    width: int
    dist: str
    alpha: float
    seed: int

    def generate(self) -> np.ndarray:
        dt = {1: np.uint8, 2: np.uint16, 4: np.uint32}[self.width]
        if self.dist == "uniform":
            return uniform(self.n, self.sigma, self.seed, dt)
        return zipf(self.n, self.sigma, self.alpha, self.seed, dt)


def batch_specs(count: int = 4096, base: int = SEED_BASE + 4, log2_min: int = 10, log2_max: int = 22,
                sigmas=(4, 20, 256, 65536), alpha: float = 1.1) -> list[SeqSpec]:
    """Batched-build workload: lengths log-uniform in [2^log2_min, 2^log2_max],
    sigma uniform over ``sigmas`` (uint8 when sigma <= 256, else uint16),
    uniform or Zipf(alpha) by a seeded coin flip."""
    x = splitmix64(base, 0, 3 * count).reshape(count, 3)
    specs = []
    span = log2_max - log2_min
    for i in range(count):
        u = float(x[i, 0] >> np.uint64(11)) / float(1 << 53)
        n = int(math.floor(2.0 ** (log2_min + span * u)))
        n = max(1 << log2_min, min(1 << log2_max, n))
        sigma = sigmas[int(x[i, 1] % np.uint64(len(sigmas)))]
        width = 1 if sigma <= 256 else 2
        dist = "zipf" if int(x[i, 2] >> np.uint64(63)) else "uniform"
        specs.append(SeqSpec(n, sigma, width, dist, alpha if dist == "zipf" else 0.0, seq_seed(base, i)))
    return specs


def serving_specs(count: int, base: int = SEED_BASE + 5, log2_min: int = 12, log2_max: int = 26,
                  sigmas=(256, 65536), alpha: float = 1.0) -> list[SeqSpec]:
    """Serving workload build requests: lengths log-uniform in [2^12, 2^26],
    sigma in {256 (uint8), 65536 (uint16)}, Zipf(1.0)."""
    x = splitmix64(base, 0, 2 * count).reshape(count, 2)
    specs = []
    span = log2_max - log2_min
    for i in range(count):
        u = float(x[i, 0] >> np.uint64(11)) / float(1 << 53)
        n = int(math.floor(2.0 ** (log2_min + span * u)))
        n = max(1 << log2_min, min(1 << log2_max, n))
        sigma = sigmas[int(x[i, 1] % np.uint64(len(sigmas)))]
        specs.append(SeqSpec(n, sigma, 1 if sigma <= 256 else 2, "zipf", alpha, seq_seed(base, i)))
    return specs
