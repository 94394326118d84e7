"""Seeded synthetic workloads (keys, values, byte strings).

This module only draws inputs. It holds none of the structure's arithmetic:
the key generator is MurmurHash3's 64-bit finalizer ``fmix64`` (Appleby),
a bijection on 64-bit words, applied to ``i ^ salt`` so that distinct indices
give distinct keys. Members use indices ``[0, n)`` and disjoint non-members
``[n, 2n)`` (or any other disjoint index range).

The paper's experiments use 64-bit integer keys (Sec. 5); the byte-string
workload (lengths uniform in 8..64, first 8 bytes a distinct 64-bit key) and
the value distributions are the synthetic recipe of this project.
"""
from __future__ import annotations

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_C1 = np.uint64(0xFF51AFD7ED558CCD)
_C2 = np.uint64(0xC4CEB9FE1A85EC53)
_S33 = np.uint64(33)


def fmix64(x: np.ndarray) -> np.ndarray:
    """MurmurHash3 fmix64 on a uint64 array (wrapping arithmetic)."""
    k = np.asarray(x, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        k ^= k >> _S33
        k *= _C1
        k ^= k >> _S33
        k *= _C2
        k ^= k >> _S33
    return k


def fmix64_scalar(x: int) -> int:
    m = (1 << 64) - 1
    x &= m
    x ^= x >> 33
    x = (x * 0xFF51AFD7ED558CCD) & m
    x ^= x >> 33
    x = (x * 0xC4CEB9FE1A85EC53) & m
    x ^= x >> 33
    return x


def key_salt(seed: int) -> int:
    """Salt XORed into the index before fmix64 (a function of the seed only)."""
    return fmix64_scalar((seed * 0x9E3779B97F4A7C15 + 0x5EED) & ((1 << 64) - 1))


def u64_keys(start: int, count: int, seed: int) -> np.ndarray:
    """Distinct 64-bit keys for indices start .. start+count-1."""
    idx = np.arange(start, start + count, dtype=np.uint64)
    return fmix64(idx ^ np.uint64(key_salt(seed)))


def values(count: int, b: int, seed: int) -> np.ndarray:
    """Uniform b-bit values (b <= 64) in the narrowest unsigned type holding b bits."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0xA11CE))
    dt = np.uint8 if b <= 8 else np.uint16 if b <= 16 else np.uint32 if b <= 32 else np.uint64
    hi = 1 << b
    return rng.integers(0, hi, size=count, dtype=np.uint64).astype(dt)


def byte_strings(start: int, count: int, seed: int, lmin: int = 8, lmax: int = 64):
    """Packed byte strings and offsets[count+1] (uint64).

    Lengths are uniform in [lmin, lmax]; the first 8 bytes of string i are the
    little-endian distinct key of index start+i, so all strings are distinct.
    """
    assert lmin >= 8
    rng = np.random.Generator(np.random.PCG64((seed << 1) ^ (start * 0x9E37) ^ 0xB17E5))
    lens = rng.integers(lmin, lmax + 1, size=count, dtype=np.int64)
    offsets = np.zeros(count + 1, dtype=np.uint64)
    np.cumsum(lens, out=offsets[1:].view(np.int64))
    total = int(offsets[-1])
    data = rng.integers(0, 256, size=total, dtype=np.uint8)
    heads = u64_keys(start, count, seed).view(np.uint8).reshape(count, 8)
    pos = offsets[:-1].astype(np.int64)
    for j in range(8):
        data[pos + j] = heads[:, j]
    return data, offsets


def log_uniform_sizes(count: int, lo: float, hi: float, seed: int) -> np.ndarray:
    """Sizes floor(10^U), U uniform in [log10 lo, log10 hi]."""
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x10C))
    u = rng.uniform(np.log10(lo), np.log10(hi), size=count)
    return np.floor(10.0 ** u).astype(np.int64)


def _signed(c: int) -> int:
    return c - (1 << 64) if c >= (1 << 63) else c


def u64_keys_torch(start: int, count: int, seed: int, device="cuda"):
    """u64_keys on a device as an int64 tensor holding the same 64-bit patterns
    (wrapping int64 arithmetic; logical shifts by masking)."""
    import torch

    k = torch.arange(start, start + count, dtype=torch.int64, device=device)
    k ^= _signed(key_salt(seed))
    m31 = (1 << 31) - 1
    k ^= (k >> 33) & m31
    k *= _signed(0xFF51AFD7ED558CCD)
    k ^= (k >> 33) & m31
    k *= _signed(0xC4CEB9FE1A85EC53)
    k ^= (k >> 33) & m31
    return k


def values_torch(count: int, b: int, seed: int, device="cuda"):
    """Uniform b-bit values on a device (narrowest unsigned dtype), seeded."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed ^ 0xA11CE)
    if b > 32:  # int64 tensor holding the 64-bit patterns
        lo = torch.randint(0, 1 << 32, (count,), dtype=torch.int64, device=device, generator=g)
        hi = torch.randint(0, 1 << (b - 32), (count,), dtype=torch.int64, device=device, generator=g)
        return lo | (hi << 32)
    v = torch.randint(0, 1 << b, (count,), dtype=torch.int64, device=device, generator=g)
    if b <= 8:
        return v.to(torch.uint8)
    if b <= 16:
        return v.to(torch.int32).to(torch.int16).view(torch.uint16)
    return v.to(torch.int64).to(torch.int32).view(torch.uint32)
