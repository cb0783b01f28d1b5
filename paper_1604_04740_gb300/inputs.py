"""Seeded synthetic inputs shared by the tests, the benchmark and the serving
driver.

This module holds none of the method's arithmetic: it only turns
(seed, tag, index) counters into pseudo-random integers with the SplitMix64
generator (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) and shapes them into the workloads the paper
measures (Sec. V): M integer streams, a shared int8 operator, job tables and
fault lists.  Everything is numpy on the host and bit-reproducible across
machines.
"""
from __future__ import annotations

import math

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TAGMUL = np.uint64(0xD1B54A32D192ED03)

# tags separating the independent random sequences of one seed
TAG_C = 1          # stream data c
TAG_G = 2          # shared operator g / G
TAG_FAULT = 3      # transient-fault positions and bits
TAG_DROP = 4       # fail-stop choices
TAG_ARRIVAL = 5    # serving arrivals
TAG_JOBS = 6       # ragged job table


def _fin(z):
    """SplitMix64 output function on a uint64 numpy array (wrapping)."""
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _key(seed: int, tag: int) -> np.uint64:
    with np.errstate(over="ignore"):
        s = _fin(np.array([seed & 0xFFFFFFFFFFFFFFFF], np.uint64) + GAMMA)
        t = np.array([tag & 0xFFFFFFFFFFFFFFFF], np.uint64) * _TAGMUL
        return _fin(s ^ t)[0]


def u64(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """count uint64 values: value i is fin(key(seed, tag) + (start + i + 1) * GAMMA)."""
    key = _key(seed, tag)
    out = np.empty(count, np.uint64)
    chunk = 1 << 22
    with np.errstate(over="ignore"):
        for b in range(0, count, chunk):
            e = min(count, b + chunk)
            ctr = np.arange(start + b + 1, start + e + 1, dtype=np.uint64)
            out[b:e] = _fin(key + ctr * GAMMA)
    return out


def int8_uniform(seed: int, tag: int, shape, start: int = 0) -> np.ndarray:
    """int8 values uniform on [-128, 127] (the low byte of each draw)."""
    n = int(np.prod(shape, dtype=np.int64))
    return (u64(seed, tag, start, n) & np.uint64(0xFF)).astype(np.uint8).view(np.int8).reshape(shape)


def int32_uniform_int8range(seed: int, tag: int, shape, start: int = 0) -> np.ndarray:
    """int32 values uniform on [-128, 127] (the paper's integer streams at the
    configured dynamic range)."""
    return int8_uniform(seed, tag, shape, start).astype(np.int32)


def int32_uniform(seed: int, tag: int, shape, lo: int, hi: int, start: int = 0) -> np.ndarray:
    """int32 values on [lo, hi] (inclusive) by v mod (hi - lo + 1); the bias is
    below 2^-32 for the ranges used here."""
    n = int(np.prod(shape, dtype=np.int64))
    span = np.uint64(hi - lo + 1)
    v = (u64(seed, tag, start, n) % span).astype(np.int64) + lo
    return v.astype(np.int32).reshape(shape)


def unit_float(seed: int, tag: int, start: int, count: int) -> np.ndarray:
    """Doubles uniform on [0, 1): the top 53 bits of each draw times 2^-53."""
    return (u64(seed, tag, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def log_uniform_int(seed: int, tag: int, start: int, count: int, lo: int, hi: int) -> np.ndarray:
    """round(exp(ln lo + U ln(hi/lo))) clamped to [lo, hi]."""
    u = unit_float(seed, tag, start, count)
    v = np.rint(np.exp(math.log(lo) + u * math.log(hi / lo))).astype(np.int64)
    return np.clip(v, lo, hi)


def _signed(v: int) -> int:
    v &= 0xFFFFFFFFFFFFFFFF
    return v - (1 << 64) if v >> 63 else v


def int8_uniform_device(seed: int, tag: int, count: int, start: int, device, chunk: int = 1 << 25):
    """The same values as int8_uniform(seed, tag, (count,), start), computed on
    a CUDA device with torch int64 arithmetic (wrapping multiply, logical
    shifts by masking).  Returns an int8 tensor."""
    import torch
    key = _signed(int(_key(seed, tag)))
    g, m1, m2 = _signed(int(GAMMA)), _signed(int(_M1)), _signed(int(_M2))
    out = torch.empty(count, dtype=torch.int8, device=device)

    def lsr(x, s):
        return (x >> s) & ((1 << (64 - s)) - 1)

    for b in range(0, count, chunk):
        e = min(count, b + chunk)
        z = torch.arange(start + b + 1, start + e + 1, dtype=torch.int64, device=device)
        z = z * g + key
        z = (z ^ lsr(z, 30)) * m1
        z = (z ^ lsr(z, 27)) * m2
        z = z ^ lsr(z, 31)
        out[b:e] = (z & 0xFF).to(torch.uint8).view(torch.int8)
    return out


# ---- workloads -------------------------------------------------------------

def streams(seed: int, shape) -> np.ndarray:
    """The M input streams c (int32 in [-128, 127])."""
    return int32_uniform_int8range(seed, TAG_C, shape)


def operator_int8(seed: int, shape) -> np.ndarray:
    """The shared operator g / G (int8 in [-128, 127])."""
    return int8_uniform(seed, TAG_G, shape)


def fault_list(seed: int, n_groups: int, n_positions: int, M: int, count: int):
    """Transient faults for the injector: `count` distinct co-located groups
    (group, position) with one flip each, a uniform stream j in [0, M) and a
    uniform bit b in [0, 63].  At most one flip per (group, position), the
    fault model under which the check is guaranteed (Prop. 4).

    Returns int64 arrays (group, position, stream, bit), sorted by
    (group, position).
    """
    total = n_groups * n_positions
    count = min(count, total)
    picked = []
    seen = set()
    start = 0
    while len(picked) < count:
        need = count - len(picked)
        cand = u64(seed, TAG_FAULT, start, 2 * need + 16) % np.uint64(total)
        start += 2 * need + 16
        for v in cand.tolist():
            if v not in seen:
                seen.add(v)
                picked.append(v)
                if len(picked) == count:
                    break
    flat = np.array(sorted(picked), np.int64)
    extra = u64(seed, TAG_FAULT + 1000, 0, 2 * count)
    j = (extra[0::2] % np.uint64(M)).astype(np.int64)
    b = (extra[1::2] % np.uint64(64)).astype(np.int64)
    return flat // n_positions, flat % n_positions, j, b
