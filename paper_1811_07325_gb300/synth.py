"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds none of the multiplication's arithmetic: it only draws
matrices.  The paper's inputs are random double matrices from Java's
``Random`` (Sec. V-A); these seeded, counter-based draws stand in for them.

Generator: SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014) used as a counter-based hash.  Element
(i, j) of matrix ``mat_id`` under ``seed`` takes the 64-bit output
``mix64(key + (c + 1) * GOLDEN)`` with ``c = i * n + j`` and
``key = mix64(seed * GOLDEN ^ (mat_id + 1) * SECOND)``, so every element can
be regenerated alone and the result does not depend on chunking or threads.

Distributions:
  * ``uniform``  : U[-1, 1): 2 * (top 53 bits / 2^53) - 1
  * ``normal``   : N(0, 1) by Box-Muller on two such uniforms (counters 2c and
                   2c + 1), z = sqrt(-2 ln(1 - u1)) * cos(2 pi u2)
  * ``int``      : integers in [lo, hi] by multiply-shift range reduction of the
                   top 32 bits
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
SECOND = np.uint64(0xD1B54A32D192ED03)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (in place on a uint64 array, which wraps mod 2^64)."""
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _key(seed: int, mat_id: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = np.array([np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * GOLDEN ^ np.uint64(mat_id + 1) * SECOND], dtype=np.uint64)
    return mix64(k)[0]


def _bits(key: np.uint64, start: int, count: int, step: int = 1, offset: int = 0) -> np.ndarray:
    c = np.arange(count, dtype=np.uint64)
    c *= np.uint64(step)
    c += np.uint64(start * step + offset + 1)
    c *= GOLDEN
    c += key
    return mix64(c)


def _fill(out: np.ndarray, fn, nthreads: int | None = None):
    flat = out.reshape(-1)
    total = flat.size
    if total == 0:
        return out
    nthreads = nthreads or min(32, os.cpu_count() or 1)
    chunk = max(1 << 20, (total + nthreads - 1) // nthreads)
    starts = list(range(0, total, chunk))
    if len(starts) == 1:
        flat[:] = fn(0, total)
        return out

    def work(s):
        e = min(total, s + chunk)
        flat[s:e] = fn(s, e - s)

    with ThreadPoolExecutor(max_workers=min(nthreads, len(starts))) as ex:
        list(ex.map(work, starts))
    return out


def uniform(n: int, seed: int, mat_id: int, dtype=np.float64, m: int | None = None) -> np.ndarray:
    """n x m (default square) matrix, entries U[-1, 1)."""
    m = n if m is None else m
    key = _key(seed, mat_id)
    out = np.empty((n, m), dtype=dtype)

    def fn(s, cnt):
        u = (_bits(key, s, cnt) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        return (2.0 * u - 1.0).astype(dtype)

    return _fill(out, fn)


def normal(n: int, seed: int, mat_id: int, dtype=np.float32, m: int | None = None) -> np.ndarray:
    """n x m (default square) matrix, entries N(0, 1) by Box-Muller."""
    m = n if m is None else m
    key = _key(seed, mat_id)
    out = np.empty((n, m), dtype=dtype)

    def fn(s, cnt):
        u1 = (_bits(key, s, cnt, step=2, offset=0) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        u2 = (_bits(key, s, cnt, step=2, offset=1) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
        r = np.sqrt(-2.0 * np.log1p(-u1))
        return (r * np.cos(2.0 * np.pi * u2)).astype(dtype)

    return _fill(out, fn)


def integers(n: int, seed: int, mat_id: int, lo: int, hi: int, m: int | None = None) -> np.ndarray:
    """n x m (default square) int64 matrix, entries uniform in [lo, hi].

    Spans up to 2^32 use multiply-shift on the top 32 bits; the full int64
    range takes the 64 bits as they are; other wide spans reduce modulo the
    span (bias below 2^-32, irrelevant here)."""
    m = n if m is None else m
    if hi < lo or lo < -2**63 or hi > 2**63 - 1:
        raise ValueError("bad range")
    span_int = hi - lo + 1
    key = _key(seed, mat_id)
    out = np.empty((n, m), dtype=np.int64)

    if span_int <= 2**32:
        span = np.uint64(span_int)

        def fn(s, cnt):
            top = _bits(key, s, cnt) >> np.uint64(32)
            return ((top * span) >> np.uint64(32)).astype(np.int64) + lo
    elif span_int == 2**64:
        def fn(s, cnt):
            return _bits(key, s, cnt).view(np.int64)
    else:
        span = np.uint64(span_int)
        lo_u = np.uint64(lo % 2**64)

        def fn(s, cnt):
            return (_bits(key, s, cnt) % span + lo_u).view(np.int64)

    return _fill(out, fn)


def sample_rows(n: int, count: int, seed: int) -> np.ndarray:
    """``count`` distinct row indices in [0, n), sorted, drawn from ``seed``."""
    count = min(count, n)
    key = _key(seed, 1_000_003)
    r = _bits(key, 0, n)
    order = np.argsort(r, kind="stable")
    return np.sort(order[:count]).astype(np.int64)


def batch_sizes(count: int, seed: int, choices=(512, 768, 1024, 1536, 2048, 3072, 4096)) -> list[int]:
    """``count`` sizes drawn uniformly from ``choices``."""
    key = _key(seed, 2_000_003)
    top = _bits(key, 0, count) >> np.uint64(32)
    idx = ((top * np.uint64(len(choices))) >> np.uint64(32)).astype(np.int64)
    return [int(choices[i]) for i in idx]


def loguniform_sizes(count: int, seed: int, lo: int, hi: int) -> list[int]:
    """``count`` integer sizes log-uniform in [lo, hi]."""
    key = _key(seed, 3_000_003)
    u = (_bits(key, 0, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    x = np.exp(np.log(lo) + u * (np.log(hi + 1) - np.log(lo)))
    return [int(min(hi, max(lo, np.floor(v)))) for v in x]


def exponential_gaps(count: int, seed: int, rate: float) -> np.ndarray:
    """``count`` inter-arrival gaps (seconds) of a Poisson stream of ``rate``/s."""
    key = _key(seed, 4_000_003)
    u = (_bits(key, 0, count) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)
    return -np.log1p(-u) / rate
