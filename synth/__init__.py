"""Seeded synthetic inputs shaped like the paper's sorting workloads.

This module holds random-number generation and workload shapes only; it
contains none of the sorting network's arithmetic.  Both the CPU oracle and
the CUDA library consume the buffers it returns.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: output i of stream `seed` is mix64(seed + (i + 1) * gamma) with
gamma = 0x9E3779B97F4A7C15 and the published mixing constants.  Because it is
counter-based it vectorises in numpy and any slice can be regenerated alone.

The paper's bitonic workload is "an input of 2^26 elements" sorted bucket by
bucket, with no distribution stated; the generators below stand in for it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

SEED_CFG1 = 0xDA2C0001
SEED_CFG2 = 0xDA2C0002
SEED_CFG3 = 0xDA2C0003
SEED_CFG4 = 0xDA2C0004
SEED_CFG5 = 0xDA2C0005


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start .. start+count-1 of the SplitMix64 stream `seed` (uint64)."""
    out = np.empty(count, dtype=np.uint64)
    chunk = 1 << 20
    s0 = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)
    with np.errstate(over="ignore"):
        for lo in range(0, count, chunk):
            hi = min(count, lo + chunk)
            z = np.arange(start + lo + 1, start + hi + 1, dtype=np.uint64)
            z *= GAMMA
            z += s0
            z ^= z >> np.uint64(30)
            z *= _M1
            z ^= z >> np.uint64(27)
            z *= _M2
            z ^= z >> np.uint64(31)
            out[lo:hi] = z
    return out


def substream(seed: int, tag: int) -> int:
    """A derived seed for an independent stream (tag-th output of `seed`)."""
    return int(splitmix64(seed ^ 0x5DEECE66D, 1, start=tag)[0])


def uniform_u32(seed: int, n: int) -> np.ndarray:
    """n uniform 32-bit words (upper halves of the 64-bit outputs)."""
    return (splitmix64(seed, n) >> np.uint64(32)).astype(np.uint32)


def uniform_u64(seed: int, n: int) -> np.ndarray:
    return splitmix64(seed, n)


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in (0, 1]: (top 53 bits + 1) * 2^-53."""
    top = (splitmix64(seed, n) >> np.uint64(11)).astype(np.float64)
    return (top + 1.0) * (1.0 / 9007199254740992.0)


def below(seed: int, n: int, bound: int) -> np.ndarray:
    """n integers in [0, bound) by multiply-shift of 32-bit words (bound < 2^32)."""
    w = uniform_u32(seed, n).astype(np.uint64)
    return ((w * np.uint64(bound)) >> np.uint64(32)).astype(np.int64)


def normal_f32(seed: int, n: int) -> np.ndarray:
    """N(0,1) by the Box-Muller transform in double precision, cast to float32."""
    half = (n + 1) // 2
    u1 = uniform01(substream(seed, 1), half)
    u2 = uniform01(substream(seed, 2), half)
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * math.pi * u2
    z = np.empty(2 * half, dtype=np.float64)
    z[0::2] = r * np.cos(t)
    z[1::2] = r * np.sin(t)
    return z[:n].astype(np.float32)


# --------------------------------------------------------------------------
# Workload shapes
# --------------------------------------------------------------------------

def cfg1_keys(seed: int = SEED_CFG1, n: int = 4096) -> np.ndarray:
    """Single-block sort: n uniform uint32 keys (4096 in the paper-sized case)."""
    return uniform_u32(seed, n)


def cfg2_kv(seed: int = SEED_CFG2, n: int = 1 << 24, skew: bool = False):
    """Key-value sort: uint32 keys (uniform, or rand mod 16 when skew) and
    payload = original index."""
    if skew:
        keys = (uniform_u32(seed, n) % np.uint32(16)).astype(np.uint32)
    else:
        keys = uniform_u32(seed, n)
    vals = np.arange(n, dtype=np.uint32)
    return keys, vals


def cfg3_f32(seed: int = SEED_CFG3, n: int = 1 << 26, dup_frac: float = 0.01,
             zeros_each: int = 4096) -> np.ndarray:
    """N(0,1) float32 keys; dup_frac of positions copy the value found at
    another random position (exact duplicates); zeros_each positions are set
    to -0.0 and as many to +0.0.  No NaN or infinity."""
    x = normal_f32(seed, n)
    ndup = int(n * dup_frac)
    if ndup:
        dst = below(substream(seed, 3), ndup, n)
        src = below(substream(seed, 4), ndup, n)
        x[dst] = x[src]
    nz = min(zeros_each, n // 4)
    if nz:
        pos = below(substream(seed, 5), 2 * nz, n)
        x[pos[:nz]] = np.float32(-0.0)
        x[pos[nz:]] = np.float32(0.0)
    return x


@dataclass
class Segments:
    keys: np.ndarray      # uint32 keys, total capacity
    vals: np.ndarray      # uint32 payload = index within segment
    offsets: np.ndarray   # uint64, num_segments + 1 (prefix sums of capacities)
    lengths: np.ndarray   # uint32 real lengths
    desc: np.ndarray      # uint8 per-segment direction (all 0 unless mixed)

    @property
    def num_segments(self) -> int:
        return int(self.lengths.size)


def next_pow2(x: np.ndarray) -> np.ndarray:
    x = np.asarray(x, dtype=np.int64)
    out = np.ones_like(x)
    m = x > 1
    out[m] = 1 << np.ceil(np.log2(x[m])).astype(np.int64)
    # guard against floating round-off at exact powers of two
    fix = out[m] // 2 >= x[m]
    out_m = out[m]
    out_m[fix] //= 2
    out[m] = out_m
    return out


def cfg4_segments(seed: int = SEED_CFG4, num_segments: int = 10000,
                  min_len: int = 32, max_len: int = 65536,
                  mixed_dirs: bool = False, largest_first: bool = False) -> Segments:
    """Independent uint32 arrays with log-uniform real lengths in
    [min_len, max_len], each stored at the next power-of-two capacity,
    laid out back to back (largest capacity first when `largest_first`, which
    puts every segment at a multiple of its capacity).  Keys are uniform in
    [0, 2^32 - 1) so that no real key equals the ascending sentinel; payload =
    index within the segment."""
    u = uniform01(substream(seed, 1), num_segments)
    lo, hi = math.log(min_len), math.log(max_len)
    lens = np.floor(np.exp(lo + (hi - lo) * u)).astype(np.int64)
    lens = np.clip(lens, min_len, max_len)
    caps = next_pow2(lens)
    if largest_first:
        order = np.argsort(-caps, kind="stable")
        lens, caps = lens[order], caps[order]
    offsets = np.zeros(num_segments + 1, dtype=np.uint64)
    offsets[1:] = np.cumsum(caps).astype(np.uint64)
    total = int(offsets[-1])
    w = uniform_u32(substream(seed, 2), total).astype(np.uint64)
    keys = ((w * np.uint64(0xFFFFFFFF)) >> np.uint64(32)).astype(np.uint32)
    vals = (np.arange(total, dtype=np.int64)
            - np.repeat(offsets[:-1].astype(np.int64), caps)).astype(np.uint32)
    if mixed_dirs:
        desc = (uniform_u32(substream(seed, 3), num_segments) & np.uint32(1)).astype(np.uint8)
    else:
        desc = np.zeros(num_segments, dtype=np.uint8)
    return Segments(keys, vals, offsets, lens.astype(np.uint32), desc)


@dataclass
class Request:
    arrival_s: float
    n: int
    desc: bool
    keys: np.ndarray   # uint64
    vals: np.ndarray   # uint32 = index


def cfg5_requests(seed: int = SEED_CFG5, count: int = 20000, min_log2: float = 8.0,
                  max_log2: float = 20.0, rate_per_s: float = 1000.0,
                  materialize: bool = True):
    """Sort requests: sizes 2^U(min_log2, max_log2) (rounded down to an
    integer length), direction Bernoulli(0.5), uint64 uniform keys, payload
    = index, Poisson arrivals at `rate_per_s` (exponential gaps)."""
    u = uniform01(substream(seed, 1), count)
    sizes = np.floor(np.exp2(min_log2 + (max_log2 - min_log2) * u)).astype(np.int64)
    sizes = np.maximum(sizes, 1)
    dirs = (uniform_u32(substream(seed, 2), count) & np.uint32(1)).astype(bool)
    gaps = -np.log(uniform01(substream(seed, 3), count)) / rate_per_s
    arrivals = np.cumsum(gaps) - gaps[0]
    out = []
    for r in range(count):
        n = int(sizes[r])
        if materialize:
            ks = uniform_u64(substream(seed, 1000 + r), n)
            vs = np.arange(n, dtype=np.uint32)
        else:
            ks = vs = None
        out.append(Request(float(arrivals[r]), n, bool(dirs[r]), ks, vs))
    return out
