"""Seeded synthetic inputs shaped like the paper's workloads.

The same bytes feed the CUDA path and the CPU oracle, so this module holds
no sorting arithmetic at all: only random draws (numpy PCG64, seed
``SEED_BASE + workload id``) and the bookkeeping to lay them out.

The paper times numpy-random decimals with 0-2 fraction digits (§6, Table 1);
the workloads below keep that recipe and scale it to GPU sizes:

* ``digits3``     u32 keys uniform in [0, 999] (a 10x10x10 cell space)
* ``u32``         u32 keys: ``uniform`` over [0, 2^32), ``zipf`` (s = 1.1 over
                  2^20 distinct values, each rank sent through a bijective
                  32-bit mixer), ``presorted`` (sorted, then a random 10% of
                  positions permuted among themselves); payload = index
* ``decimal``     int64 fixed-point decimals, 6 integer + 3 fraction digits,
                  stored scaled by 1000, sign +/- with probability 1/2
* ``strings``     lowercase ASCII strings, lengths uniform in 1..16, packed
                  into one char buffer plus n+1 uint32 offsets
* ``segments``    uneven segments: sizes log-uniform in [16, 2^20]
* ``rows``        float32 rows of distinct keys: a permutation of 0..L-1 plus
                  a per-row offset in [0, 0.5)
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 20210703

WORKLOAD_IDS = {"digits3": 0, "u32": 1, "decimal": 2, "strings": 3, "segments": 4, "rows": 5}


def rng_for(workload: str, extra: int = 0) -> np.random.Generator:
    return np.random.default_rng(SEED_BASE + WORKLOAD_IDS[workload] + 1000 * extra)


def mix32(x: np.ndarray) -> np.ndarray:
    """A bijective 32-bit mixer (the MurmurHash3 32-bit finaliser)."""
    x = np.asarray(x, dtype=np.uint32).copy()
    x ^= x >> np.uint32(16)
    x *= np.uint32(0x85EBCA6B)
    x ^= x >> np.uint32(13)
    x *= np.uint32(0xC2B2AE35)
    x ^= x >> np.uint32(16)
    return x


def digits3(n: int, seed_extra: int = 0) -> np.ndarray:
    """u32 keys uniform in [0, 999]: three base-10 digit dimensions."""
    return rng_for("digits3", seed_extra).integers(0, 1000, n, dtype=np.uint32)


def zipf_ranks(rng: np.random.Generator, n: int, s: float = 1.1,
               distinct: int = 1 << 20) -> np.ndarray:
    """Ranks in [1, distinct] with P(r) proportional to r^-s (inverse CDF)."""
    r = np.arange(1, distinct + 1, dtype=np.float64)
    cdf = np.cumsum(r ** -s)
    cdf /= cdf[-1]
    u = rng.random(n)
    try:  # multi-threaded binary search; identical result to numpy's
        import torch
        idx = torch.searchsorted(torch.from_numpy(cdf), torch.from_numpy(u), right=True).numpy()
    except ImportError:  # pragma: no cover
        idx = np.searchsorted(cdf, u, side="right")
    return np.minimum(idx, distinct - 1).astype(np.uint32) + np.uint32(1)


def u32_keys(n: int, dist: str = "uniform", seed_extra: int = 0) -> np.ndarray:
    rng = rng_for("u32", seed_extra)
    if dist == "uniform":
        return rng.integers(0, 1 << 32, n, dtype=np.uint32)
    if dist == "zipf":
        return mix32(zipf_ranks(rng, n))
    if dist == "presorted":
        a = np.sort(rng.integers(0, 1 << 32, n, dtype=np.uint32))
        sel = np.nonzero(rng.random(n) < 0.10)[0]
        a[sel] = a[rng.permutation(sel)]
        return a
    raise ValueError(f"unknown distribution {dist!r}")


def u32_pairs(n: int, dist: str = "uniform", seed_extra: int = 0):
    """(keys, payload) with payload = input index (uint32)."""
    return u32_keys(n, dist, seed_extra), np.arange(n, dtype=np.uint32)


def u64_keys(n: int, seed_extra: int = 0) -> np.ndarray:
    rng = rng_for("u32", 7 + seed_extra)
    return rng.integers(0, np.iinfo(np.uint64).max, n, dtype=np.uint64, endpoint=True)


def decimals(n: int, int_digits: int = 6, frac_digits: int = 3, seed_extra: int = 0):
    """int64 = sign * m with m uniform in [0, 10^(int+frac)), sign 50/50."""
    rng = rng_for("decimal", seed_extra)
    m = rng.integers(0, 10 ** (int_digits + frac_digits), n, dtype=np.int64)
    sign = rng.integers(0, 2, n, dtype=np.int64) * 2 - 1
    return sign * m


def strings(n: int, min_len: int = 1, max_len: int = 16, lo: int = 97, hi: int = 123,
            seed_extra: int = 0):
    """(chars uint8, offsets uint32[n+1]) of n strings over bytes [lo, hi)."""
    rng = rng_for("strings", seed_extra)
    lens = rng.integers(min_len, max_len + 1, n, dtype=np.int64)
    offsets = np.zeros(n + 1, np.int64)
    np.cumsum(lens, out=offsets[1:])
    chars = rng.integers(lo, hi, int(offsets[-1]), dtype=np.uint8)
    return chars, offsets.astype(np.uint32)


def segment_sizes(num_segments: int = 65536, lo: int = 16, hi: int = 1 << 20,
                  total: int | None = None, seed_extra: int = 0) -> np.ndarray:
    """Log-uniform sizes in [lo, hi]; if total is given, rescaled to sum to it."""
    rng = rng_for("segments", seed_extra)
    sizes = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), num_segments))).astype(np.int64)
    if total is not None:
        sizes = np.maximum(np.rint(sizes * (total / sizes.sum())).astype(np.int64), 1)
        big = int(np.argmax(sizes))  # the rounding error goes to the largest segment
        sizes[big] += total - sizes.sum()
        if sizes[big] < 1:
            raise ValueError("total too small for the number of segments")
    return sizes


def segments(sizes: np.ndarray, seed_extra: int = 0):
    """(u32 keys, f32 values, u64 offsets[num+1]) for the given segment sizes."""
    rng = rng_for("segments", 100 + seed_extra)
    n = int(sizes.sum())
    keys = rng.integers(0, 1 << 32, n, dtype=np.uint32)
    vals = rng.standard_normal(n, dtype=np.float32)
    offsets = np.zeros(sizes.size + 1, np.uint64)
    np.cumsum(sizes, out=offsets[1:])
    return keys, vals, offsets


def distinct_rows(rows: int, length: int, seed_extra: int = 0) -> np.ndarray:
    """float32 rows: a permutation of 0..L-1 plus a per-row offset in [0, 0.5)."""
    rng = rng_for("rows", seed_extra)
    x = np.empty((rows, length), np.float32)
    for r in range(rows):
        x[r] = rng.permutation(length).astype(np.float32) + np.float32(rng.uniform(0, 0.5))
    return x
