"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle's
callers.  This module holds none of the dispatch method's arithmetic: it only
draws numbers.

Host arrays come from a counter-based SplitMix64 stream (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014): output
i of stream (seed, key) is the SplitMix64 finaliser applied to
``base + (i + 1) * 0x9E3779B97F4A7C15`` where ``base`` is the finaliser of a
mix of seed and key.  Any slice of a stream can be generated on its own.

Large device pools (gigabytes, used only by the benchmark) come from torch's
seeded device generator instead; items drawn from them are copied back to the
host whenever the oracle checks them.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _fin(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def stream_base(seed: int, key: int) -> np.uint64:
    x = np.array([(seed * 0x632BE59BD9B4E019 + key * 0xD6E8FEB86659FD93) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
    return _fin(x)[0]


def u64(seed: int, key: int, n: int, offset: int = 0) -> np.ndarray:
    """n uniform 64-bit words: outputs offset .. offset+n-1 of stream (seed, key)."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        return _fin(stream_base(seed, key) + i * GOLDEN)


def int32_uniform(seed: int, key: int, n: int, lo: int, hi: int) -> np.ndarray:
    """Integers uniform on [lo, hi] (multiply-shift on the high 32 bits)."""
    span = np.uint64(hi - lo + 1)
    u = u64(seed, key, n) >> np.uint64(32)
    return (np.int64(lo) + ((u * span) >> np.uint64(32)).astype(np.int64)).astype(np.int32)


def bytes_uniform(seed: int, key: int, n: int) -> np.ndarray:
    """n bytes uniform on 0..255 (the 8 bytes of each word, little-endian)."""
    w = u64(seed, key, (n + 7) // 8)
    return w.view(np.uint8)[:n].copy()


def unit_open(seed: int, key: int, n: int) -> np.ndarray:
    """Doubles uniform on (0, 1]: (top 53 bits + 1) * 2^-53."""
    return ((u64(seed, key, n) >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)


def normal_f32(seed: int, key: int, n: int) -> np.ndarray:
    """Standard normal float32 by the Box-Muller transform."""
    u1 = unit_open(seed, key, n)
    u2 = unit_open(seed, key ^ 0x5bd1e995, n)
    return (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)).astype(np.float32)


def exponential(seed: int, key: int, n: int, mean: float) -> np.ndarray:
    """Exponential inter-arrival gaps with the given mean (Poisson arrivals)."""
    return -np.log(unit_open(seed, key, n)) * mean


def log_uniform_int(seed: int, key: int, n: int, lo: int, hi: int) -> np.ndarray:
    """Integers whose logarithm is uniform on [log lo, log hi]."""
    u = unit_open(seed, key, n)
    v = np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))
    return np.clip(np.floor(v), lo, hi).astype(np.int64)


def choice(seed: int, key: int, n: int, k: int) -> np.ndarray:
    """Integers uniform on 0..k-1."""
    u = u64(seed, key, n) >> np.uint64(32)
    return ((u * np.uint64(k)) >> np.uint64(32)).astype(np.int64)


def permutation(seed: int, key: int, n: int) -> np.ndarray:
    """A permutation of 0..n-1 (sort of n random words)."""
    return np.argsort(u64(seed, key, n), kind="stable")


# ---- device pools (torch, seeded) ---------------------------------------------------
def device_pool(kind: str, nbytes: int, seed: int, device: str = "cuda"):
    """A device tensor of `nbytes` bytes of seeded synthetic data.
    kind: "i32" (uniform [-2^20, 2^20]), "u8" (uniform bytes), "f32" (N(0,1))."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    if kind == "i32":
        return torch.randint(-(1 << 20), (1 << 20) + 1, (nbytes // 4,), dtype=torch.int32, device=device, generator=g)
    if kind == "u8":
        return torch.randint(0, 256, (nbytes,), dtype=torch.uint8, device=device, generator=g)
    if kind == "f32":
        return torch.randn((nbytes // 4,), dtype=torch.float32, device=device, generator=g)
    raise ValueError(kind)
