"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module holds no transform arithmetic: it only turns (seed, stream, index)
into integers uniform in [0, m), and draws the length mixes of the batched
workloads.  The generator is counter based, so any element can be regenerated
independently:

    key(seed, stream)  = mix64(seed * G + stream)
    draw(i, attempt)   = mix64(key + (i * 64 + attempt) * G)          (mod 2^64)
    value_i            = the first draw(i, a), a = 0, 1, ..., whose low
                         bitlen(m) bits are < m   (mask-and-reject)

mix64 is the SplitMix64 output finaliser (Steele, Lea, Flood, OOPSLA 2014):
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9; z ^= z >> 27; z *= 0x94D049BB133111EB; z ^= z >> 31
and G = 0x9E3779B97F4A7C15.  Mask-and-reject gives exactly uniform values.
"""
from __future__ import annotations

import numpy as np

G = np.uint64(0x9E3779B97F4A7C15)
_C1 = np.uint64(0xBF58476D1CE4E5B9)
_C2 = np.uint64(0x94D049BB133111EB)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser on a uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=np.uint64).copy()
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _C1
        z ^= z >> np.uint64(27)
        z *= _C2
        z ^= z >> np.uint64(31)
    return z


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = np.array([seed], dtype=np.uint64) * G + np.uint64(stream)
    return mix64(k)[0]


def uniform_mod(m: int, count: int, seed: int, stream: int, start: int = 0,
                dtype=np.uint32, chunk: int = 1 << 24) -> np.ndarray:
    """``count`` values uniform in [0, m), elements ``start .. start+count-1``
    of stream ``(seed, stream)``."""
    if m < 1:
        raise ValueError("m must be >= 1")
    bits = max(1, int(m - 1).bit_length())
    mask = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    key = _key(seed, stream)
    out = np.empty(count, dtype=dtype)
    for c0 in range(0, count, chunk):
        n = min(chunk, count - c0)
        idx = np.arange(start + c0, start + c0 + n, dtype=np.uint64)
        vals = np.empty(n, dtype=np.uint64)
        todo = np.arange(n)
        attempt = 0
        while todo.size:
            if attempt >= 64:
                raise RuntimeError("rejection sampling did not terminate")
            with np.errstate(over="ignore"):
                ctr = key + (idx[todo] * np.uint64(64) + np.uint64(attempt)) * G
            v = mix64(ctr) & mask
            ok = v < np.uint64(m)
            vals[todo[ok]] = v[ok]
            todo = todo[~ok]
            attempt += 1
        out[c0:c0 + n] = vals.astype(dtype)
    return out


def pairs(m: int, batch: int, N: int, seed: int, dtype=np.uint32):
    """(f, g) of shape [batch, N], uniform in [0, m); f is stream 0, g stream 1."""
    f = uniform_mod(m, batch * N, seed, 0, dtype=dtype).reshape(batch, N)
    g = uniform_mod(m, batch * N, seed, 1, dtype=dtype).reshape(batch, N)
    return f, g


def log_uniform_lengths(count: int, lo_log2: int, hi_log2: int, seed: int, stream: int = 7) -> np.ndarray:
    """``count`` lengths 2^k with k uniform on {lo_log2 .. hi_log2} (the uneven
    batch and the serving mix)."""
    k = uniform_mod(hi_log2 - lo_log2 + 1, count, seed, stream, dtype=np.uint64)
    return (np.uint64(1) << (k + np.uint64(lo_log2))).astype(np.int64)


def exponential_gaps(count: int, rate_per_s: float, seed: int, stream: int = 9) -> np.ndarray:
    """Poisson-process inter-arrival gaps in seconds: -ln(U)/rate with U uniform
    in (0, 1] built from 53-bit draws of the same generator."""
    u53 = uniform_mod(1 << 53, count, seed, stream, dtype=np.uint64).astype(np.float64)
    u = (u53 + 1.0) / float(1 << 53)
    return -np.log(u) / rate_per_s


# ---- the same generator in torch (device-side generation of large inputs) ----

def _torch_consts():
    import torch

    def s64(v):  # uint64 constant as the int64 with the same bits
        return torch.tensor(v - (1 << 64) if v >= (1 << 63) else v, dtype=torch.int64)
    return s64


def _lsr(t, s):
    """Logical right shift of int64 bit patterns."""
    import torch
    return (t >> s) & ((1 << (64 - s)) - 1)


def mix64_torch(z):
    """SplitMix64 finaliser on int64 tensors holding uint64 bit patterns."""
    s64 = _torch_consts()
    c1, c2 = s64(0xBF58476D1CE4E5B9).to(z.device), s64(0x94D049BB133111EB).to(z.device)
    z = z ^ _lsr(z, 30)
    z = z * c1
    z = z ^ _lsr(z, 27)
    z = z * c2
    return z ^ _lsr(z, 31)


def uniform_mod_torch(m: int, count: int, seed: int, stream: int, start: int = 0, device="cuda",
                      dtype=None, chunk: int = 1 << 26):
    """``uniform_mod`` computed with torch on ``device``: identical values."""
    import torch
    s64 = _torch_consts()
    bits = max(1, int(m - 1).bit_length())
    mask = (1 << bits) - 1
    key = int(_key(seed, stream))
    key_t = s64(key).to(device)
    g_t = s64(int(G)).to(device)
    out_dtype = dtype or (torch.int32 if m <= (1 << 31) else torch.int64)
    out = torch.empty(count, dtype=out_dtype, device=device)
    for c0 in range(0, count, chunk):
        n = min(chunk, count - c0)
        idx = torch.arange(start + c0, start + c0 + n, dtype=torch.int64, device=device)
        vals = torch.empty(n, dtype=torch.int64, device=device)
        todo = torch.arange(n, device=device)
        attempt = 0
        while todo.numel():
            if attempt >= 64:
                raise RuntimeError("rejection sampling did not terminate")
            ctr = key_t + (idx[todo] * 64 + attempt) * g_t
            v = mix64_torch(ctr)
            v = v & mask if bits < 64 else v
            ok = (v >= 0) & (v < m) if bits < 64 else v.to(torch.float64) < float(m)
            vals[todo[ok]] = v[ok]
            todo = todo[~ok]
            attempt += 1
        out[c0:c0 + n] = vals.to(out_dtype)
    return out
