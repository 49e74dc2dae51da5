"""Seeded synthetic inputs shaped like the paper's key-only workloads.

This module only *draws* inputs: key columns, row-ids, probe sides, query sizes
and arrival times.  It holds none of the arithmetic of the method (no key
transform, no selection, no hashing), so the CPU oracle and the CUDA path can
both be fed from it without sharing any of the code under test.

Random numbers come from counter-based splitmix64 (G. L. Steele, D. Lea,
C. H. Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
``x_i = mix(seed + (i + 1) * GAMMA)`` with the published mix constants.  A
workload seed ``s`` owns sub-streams ``s * 16 + j`` (j = 0 keys, 1 distinct
values, 2 choices, 3 hit coins, 4 hit picks, 5 miss draws, 6 permutation,
7 multiplicities, 8 sizes, 9 extra), so every array is reproducible from
(seed, j, index) alone, on any machine and in any chunking.

The paper's own data (a PostgreSQL table of ``value double, payload text``,
Sec. V-A) and its scripts are not published; these generators stand in for it
with the shapes of the paper's workloads: wide key columns with (key, row-id)
pairs, Top-K with small K, and a hash join whose build side is a key column.
"""
from __future__ import annotations

import concurrent.futures as _cf
import os

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22
_U64 = np.uint64


def stream_seed(seed: int, j: int) -> int:
    """Seed of sub-stream ``j`` of workload seed ``seed``."""
    return (int(seed) * 16 + int(j)) & 0xFFFFFFFFFFFFFFFF


def _mix(z: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        z = (z ^ (z >> _U64(30))) * _M1
        z = (z ^ (z >> _U64(27))) * _M2
        return z ^ (z >> _U64(31))


def _fill(out: np.ndarray, seed: int, start: int) -> None:
    i = np.arange(start + 1, start + 1 + out.shape[0], dtype=np.uint64)
    with np.errstate(over="ignore"):
        out[:] = _mix(_U64(seed) + i * _U64(GAMMA))


def _threads() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def _par_chunks(count: int, fn) -> None:
    """Call ``fn(a, b)`` over [0, count) in chunks, on a thread pool for large
    counts (numpy's searches and gathers release the interpreter lock)."""
    count = int(count)
    if count <= _CHUNK:
        if count:
            fn(0, count)
        return
    spans = [(a, min(a + _CHUNK, count)) for a in range(0, count, _CHUNK)]
    with _cf.ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(lambda ab: fn(*ab), spans))


def _searchsorted(sorted_a: np.ndarray, v: np.ndarray, side: str = "left") -> np.ndarray:
    out = np.empty(v.shape[0], dtype=np.int64)

    def part(a, b):
        out[a:b] = np.searchsorted(sorted_a, v[a:b], side=side)
    _par_chunks(v.shape[0], part)
    return out


def _take(src: np.ndarray, idx: np.ndarray) -> np.ndarray:
    out = np.empty(idx.shape[0], dtype=src.dtype)

    def part(a, b):
        out[a:b] = src[idx[a:b]]
    _par_chunks(idx.shape[0], part)
    return out


def splitmix64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """``count`` uint64 draws x_start .. x_{start+count-1} of stream ``seed``."""
    out = np.empty(int(count), dtype=np.uint64)
    if count <= _CHUNK:
        _fill(out, seed, start)
        return out
    spans = [(a, min(a + _CHUNK, count)) for a in range(0, count, _CHUNK)]
    with _cf.ThreadPoolExecutor(_threads()) as ex:
        list(ex.map(lambda ab: _fill(out[ab[0]:ab[1]], seed, start + ab[0]), spans))
    return out


def _i64(v: int) -> int:
    v &= 0xFFFFFFFFFFFFFFFF
    return v - (1 << 64) if v >> 63 else v


def splitmix64_torch(seed: int, count: int, start: int = 0, device="cuda", chunk: int = 1 << 26):
    """The same draws as ``splitmix64`` as a torch int64 tensor (bit-identical),
    computed on ``device`` with wrapping int64 arithmetic (logical shifts are
    an arithmetic shift and a mask)."""
    import torch
    out = torch.empty(int(count), dtype=torch.int64, device=device)
    g, m1, m2 = _i64(GAMMA), _i64(0xBF58476D1CE4E5B9), _i64(0x94D049BB133111EB)
    s0 = _i64(seed)

    def lsr(x, k):
        return (x >> k) & ((1 << (64 - k)) - 1)

    for a in range(0, int(count), chunk):
        b = min(int(count), a + chunk)
        i = torch.arange(start + a + 1, start + b + 1, dtype=torch.int64, device=device)
        z = i * g + s0
        z = (z ^ lsr(z, 30)) * m1
        z = (z ^ lsr(z, 27)) * m2
        out[a:b] = z ^ lsr(z, 31)
    return out


def unit_f64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each draw."""
    out = np.empty(int(count), dtype=np.float64)

    def part(a, b):
        raw = np.empty(b - a, dtype=np.uint64)
        _fill(raw, seed, start + a)
        out[a:b] = (raw >> _U64(11)).astype(np.float64) * (1.0 / (1 << 53))
    _par_chunks(count, part)
    return out


def log_uniform(lo: float, hi: float, seed: int, count: int) -> np.ndarray:
    """``floor(lo * (hi / lo) ** u)`` with u uniform in [0, 1); int64."""
    u = unit_f64(seed, count)
    return np.floor(lo * np.power(hi / lo, u)).astype(np.int64)


# --------------------------------------------------------------------------
# Top-K key columns
# --------------------------------------------------------------------------

def _distinct_u64(seed: int, count: int) -> np.ndarray:
    """``count`` distinct draws of stream ``seed`` in draw order (redraw dups)."""
    got = splitmix64(seed, count)
    nxt = count
    while True:
        _, first = np.unique(got, return_index=True)
        if first.shape[0] == count:
            return got
        keep = np.zeros(count, dtype=bool)
        keep[first] = True
        bad = np.flatnonzero(~keep)
        got[bad] = splitmix64(seed, bad.shape[0], start=nxt)
        nxt += bad.shape[0]


def _ascending_f32_bits(n: int) -> np.ndarray:
    """Strictly increasing finite float32 values, negatives then non-negatives.

    IEEE 754 encodes a non-negative finite float so that a larger magnitude has
    a larger bit pattern; the sign bit makes it negative.  The first half are
    negative values of falling magnitude, the second half non-negative values of
    rising magnitude, all below the infinity pattern 0x7F800000.
    """
    neg = n // 2
    pos = n - neg
    stride = max(1, 0x7F800000 // max(1, max(neg, pos)))
    out = np.empty(n, dtype=np.uint32)
    out[:neg] = np.uint32(0x80000000) | ((neg - np.arange(neg, dtype=np.uint64)) * stride).astype(np.uint32)
    out[neg:] = (np.arange(pos, dtype=np.uint64) * stride).astype(np.uint32)
    return out


def _ascending_f64_bits(n: int) -> np.ndarray:
    """Strictly increasing finite float64 values, negatives then non-negatives
    (the binary64 counterpart of ``_ascending_f32_bits``)."""
    neg = n // 2
    pos = n - neg
    stride = max(1, 0x7FF0000000000000 // max(1, max(neg, pos)))
    out = np.empty(n, dtype=np.uint64)
    with np.errstate(over="ignore"):
        out[:neg] = _U64(1 << 63) | ((neg - np.arange(neg, dtype=np.uint64)) * _U64(stride))
        out[neg:] = np.arange(pos, dtype=np.uint64) * _U64(stride)
    return out


_DTYPE = {"i64": np.int64, "f32": np.float32, "f64": np.float64, "u64": np.uint64, "i32": np.int32,
          "u32": np.uint32}


def topk_keys(n: int, dist: str = "uniform", key_type: str = "i64", seed: int = 0) -> np.ndarray:
    """A key column of ``n`` keys of type ``key_type`` (i64, f32, f64, u64,
    i32, u32).

    dist:
      * ``uniform``: uniform bit patterns of the type's width (integers over
        their full range; floats over all classes: NaN, inf, subnormal, +-0).
      * ``ascending``: strictly increasing.  int64: ``INT64_MIN + i*floor(2^64/n)``,
        uint64 the same offset by 2^63, 32-bit integers likewise over 2^32 (for
        n <= 2^32); floats: see ``_ascending_f32_bits`` / ``_ascending_f64_bits``.
      * ``dup1024``: each key one of 1024 distinct uniform draws, picked by a
        second stream.
    """
    n = int(n)
    if key_type not in _DTYPE:
        raise ValueError(key_type)
    wide = key_type in ("i64", "f64", "u64")
    dt = _DTYPE[key_type]
    if dist == "uniform":
        raw = splitmix64(stream_seed(seed, 0), n)
        if wide:
            return raw.view(dt)
        return (raw >> _U64(32)).astype(np.uint32).view(dt)
    if dist == "ascending":
        if key_type == "f64":
            return _ascending_f64_bits(n).view(np.float64)
        if key_type == "f32":
            return _ascending_f32_bits(n).view(np.float32)
        span = 1 << (64 if wide else 32)
        step = min(span // max(n, 1), span - 1)          # n = 1: only i = 0 is used
        with np.errstate(over="ignore"):
            v = np.arange(n, dtype=np.uint64) * _U64(step)
        if wide:
            return (v + _U64(1 << 63)).view(np.int64) if key_type == "i64" else v.view(dt)
        v32 = v.astype(np.uint32)
        return (v32 ^ np.uint32(1 << 31)).view(np.int32) if key_type == "i32" else v32
    if dist == "dup1024":
        if wide:
            vals = _distinct_u64(stream_seed(seed, 1), 1024).view(dt)
        else:
            bits = (splitmix64(stream_seed(seed, 1), 4096) >> _U64(32)).astype(np.uint32)
            _, first = np.unique(bits, return_index=True)
            vals = bits[np.sort(first)[:1024]].view(dt)
            assert vals.shape[0] == 1024
        pick = splitmix64(stream_seed(seed, 2), n) % _U64(1024)
        return vals[pick.astype(np.int64)]
    raise ValueError(dist)


def identity_rowids(n: int) -> np.ndarray:
    return np.arange(int(n), dtype=np.uint32)


# --------------------------------------------------------------------------
# Hash-join sides
# --------------------------------------------------------------------------

class JoinBuild:
    """Build side: ``keys`` (int64) with row-ids ``0..n-1``, the distinct keys
    and how many rows carry each of them (``mult``, aligned with ``distinct``)."""

    def __init__(self, keys: np.ndarray, distinct: np.ndarray, mult: np.ndarray):
        self.keys = keys
        self.rowids = identity_rowids(keys.shape[0])
        self.distinct = distinct
        self.mult = mult


def join_build(n: int, mult: str = "unique", seed: int = 2) -> JoinBuild:
    """``n`` build rows.  ``unique``: all keys distinct.  ``mult14``: distinct
    keys each repeated m ~ U{1..4} times (the last truncated so the total is
    exactly n), rows shuffled by a seeded permutation."""
    n = int(n)
    if mult == "unique":
        keys = _distinct_u64(stream_seed(seed, 1), n).view(np.int64)
        return JoinBuild(keys, keys, np.ones(n, dtype=np.int64))
    if mult != "mult14":
        raise ValueError(mult)
    m = (splitmix64(stream_seed(seed, 7), n) % _U64(4)).astype(np.int64) + 1
    csum = np.cumsum(m)
    d = int(np.searchsorted(csum, n)) + 1          # distinct keys needed
    m = m[:d].copy()
    m[-1] -= int(csum[d - 1]) - n
    distinct = _distinct_u64(stream_seed(seed, 1), d).view(np.int64)
    rows = np.repeat(distinct, m)
    perm = np.argsort(splitmix64(stream_seed(seed, 6), n), kind="stable")
    return JoinBuild(rows[perm], distinct, m)


def _zipf_ranks(u: np.ndarray, d: int, s: float) -> np.ndarray:
    """Inverse-CDF draw of ranks 0..d-1 with P(rank r) proportional to (r+1)^-s."""
    w = np.power(np.arange(1, d + 1, dtype=np.float64), -s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    r = _searchsorted(cdf, u, side="right")
    return np.minimum(r, d - 1)


class JoinProbe:
    def __init__(self, keys: np.ndarray, hit: np.ndarray, pick: np.ndarray):
        self.keys = keys
        self.hit = hit                   # bool per probe row: drawn as a hit
        self.pick = pick                 # index into the build's distinct keys (hits only)
        self.rowids = identity_rowids(keys.shape[0])

    def expected_pairs(self, build: "JoinBuild") -> int:
        """Pairs the join must return: the build multiplicity of every hit."""
        return int(build.mult[self.pick[self.hit]].sum())


def join_probe(n: int, build: JoinBuild, hit_rate: float = 0.9, dist: str = "uniform",
               seed: int = 2, zipf_s: float = 1.1) -> JoinProbe:
    """``n`` probe keys.  Each row is a hit with probability ``hit_rate``; a hit
    draws one of the build side's distinct keys (uniformly, or Zipf(s) by rank
    over a seeded permutation of the distinct keys); a miss draws a uniform
    int64 that is not a build key."""
    n = int(n)
    d = build.distinct.shape[0]
    hit = unit_f64(stream_seed(seed, 3), n) < hit_rate
    u = unit_f64(stream_seed(seed, 4), n)
    if dist == "uniform":
        idx = np.empty(n, dtype=np.int64)

        def part(a, b):
            idx[a:b] = np.minimum(np.floor(u[a:b] * d).astype(np.int64), d - 1)
        _par_chunks(n, part)
    elif dist == "zipf":
        ranks = _zipf_ranks(u, d, zipf_s)
        perm = np.argsort(splitmix64(stream_seed(seed, 6), d), kind="stable")
        idx = _take(perm, ranks)
    else:
        raise ValueError(dist)
    keys = _take(build.distinct, idx)
    nm = int(n - int(hit.sum()))
    miss = splitmix64(stream_seed(seed, 5), nm).view(np.int64)
    sorted_build = np.sort(build.distinct)
    nxt = nm
    while nm:
        pos = np.minimum(_searchsorted(sorted_build, miss), d - 1)
        bad = np.flatnonzero(_take(sorted_build, pos) == miss)
        if bad.shape[0] == 0:
            break
        miss[bad] = splitmix64(stream_seed(seed, 5), bad.shape[0], start=nxt).view(np.int64)
        nxt += bad.shape[0]
    keys[~hit] = miss
    return JoinProbe(keys, hit, idx)


# --------------------------------------------------------------------------
# Batched and serving workloads
# --------------------------------------------------------------------------

def batched_topk_queries(count: int = 4096, lo: float = 1e3, hi: float = 4e6,
                         kmax: int = 1000, seed: int = 3):
    """Sizes N ~ logU[lo, hi) and K ~ U{1..kmax} of a batch of Top-K queries."""
    ns = log_uniform(lo, hi, stream_seed(seed, 8), count)
    ks = (splitmix64(stream_seed(seed, 9), count) % _U64(kmax)).astype(np.int64) + 1
    return ns, ks


def batched_probe_sizes(count: int = 1024, lo: float = 1e3, hi: float = 1e6, seed: int = 3):
    return log_uniform(lo, hi, stream_seed(seed, 10), count)


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 4) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process of rate ``rate_per_s``."""
    u = unit_f64(stream_seed(seed, 11), count)
    gaps = -np.log1p(-u) / rate_per_s
    return np.cumsum(gaps)
