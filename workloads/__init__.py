"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no cipher arithmetic: it only turns (seed, stream, count) into
bytes with SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014), used as a counter-based generator: output i of a
stream is mix(base + (i + 1) * GAMMA), so any slice can be produced without
generating what comes before it.

Workload recipes (sizes, key mixes, request-size distributions) live here too, so
that the oracle side and the CUDA side see byte-identical inputs.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# Stream ids: one independent sequence per kind of input drawn from a seed.
STREAM_DATA = 1
STREAM_KEY = 2
STREAM_IV = 3
STREAM_REQ = 4
STREAM_ARRIVAL = 5


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def _base(seed: int, stream: int) -> np.uint64:
    s = np.array([(seed & 0xFFFFFFFF) << 32 | (stream & 0xFFFFFFFF)], dtype=np.uint64)
    return _mix(s)[0]


def u64(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """Words start .. start+n-1 of the (seed, stream) sequence, as uint64."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        return _mix(_base(seed, stream) + i * GAMMA)


def seeded_bytes(seed: int, stream: int, nbytes: int) -> np.ndarray:
    """nbytes uniform random bytes (little-endian bytes of consecutive words)."""
    nwords = (nbytes + 7) // 8
    out = np.empty(nwords, dtype=np.uint64)
    chunk = 1 << 24
    for w0 in range(0, nwords, chunk):
        n = min(chunk, nwords - w0)
        out[w0:w0 + n] = u64(seed, stream, n, start=w0)
    return out.view(np.uint8)[:nbytes].copy() if nbytes % 8 else out.view(np.uint8)


def uniform01(seed: int, stream: int, n: int) -> np.ndarray:
    """n doubles in [0, 1) from the top 53 bits of each word."""
    return (u64(seed, stream, n) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def xts_key(seed: int, key_bits: int, index: int = 0) -> bytes:
    """K1 || K2 for AES-key_bits-XTS (2 * key_bits / 8 bytes). K1 != K2 always holds
    for these draws (checked, so a collision would fail loudly, never silently)."""
    nb = key_bits // 8
    raw = seeded_bytes(seed, STREAM_KEY, 64 * (index + 1))[64 * index: 64 * index + 2 * nb]
    k = bytes(raw)
    if k[:nb] == k[nb:]:
        raise ValueError("seeded XTS key halves collide")
    return k


def single_key(seed: int, key_bits: int, index: int = 0) -> bytes:
    nb = key_bits // 8
    raw = seeded_bytes(seed, STREAM_KEY, 64 * (index + 1))[64 * index: 64 * index + nb]
    return bytes(raw)


def page_ivs(seed: int, npages: int) -> np.ndarray:
    """One 16-byte IV per page, shape (npages, 16), uint8."""
    return seeded_bytes(seed, STREAM_IV, 16 * npages).reshape(npages, 16)


# ---------------------------------------------------------------------------
# Request mixes (batched and serving workloads)
# ---------------------------------------------------------------------------

MODE_XTS = 0
MODE_CBC_DEC = 1
MODE_CBC_ENC = 2
MODE_ECB = 3


@dataclass
class RequestMix:
    sizes: np.ndarray      # bytes, multiples of 4096
    modes: np.ndarray      # MODE_* per request
    dirs: np.ndarray       # 0 encrypt / 1 decrypt (XTS and ECB only)
    keys: np.ndarray       # key index per request
    key_bits: np.ndarray   # per key: 128 or 256
    offsets: np.ndarray    # byte offset of each request in one packed buffer

    @property
    def total_bytes(self) -> int:
        return int(self.sizes.sum())


def log_uniform_pages(u: np.ndarray, lo: int, hi: int, page: int = 4096) -> np.ndarray:
    """size = page * max(1, round(exp(U(ln lo, ln hi)) / page))."""
    s = np.exp(np.log(lo) + u * (np.log(hi) - np.log(lo)))
    return (page * np.maximum(1, np.rint(s / page))).astype(np.int64)


def request_mix(seed: int, n: int, lo: int, hi: int, nkeys: int,
                mode_split=(0.5, 0.25, 0.25)) -> RequestMix:
    """n requests, sizes log-uniform in [lo, hi] rounded to 4 KiB pages, nkeys keys
    (first half AES-128, second half AES-256), modes XTS / CBC-dec / CBC-enc drawn
    with the given split; XTS direction drawn 50/50."""
    u = uniform01(seed, STREAM_REQ, 4 * n).reshape(n, 4)
    sizes = log_uniform_pages(u[:, 0], lo, hi)
    c1 = mode_split[0]
    c2 = mode_split[0] + mode_split[1]
    modes = np.where(u[:, 1] < c1, MODE_XTS, np.where(u[:, 1] < c2, MODE_CBC_DEC, MODE_CBC_ENC))
    dirs = (u[:, 2] < 0.5).astype(np.int32)
    keys = np.minimum((u[:, 3] * nkeys).astype(np.int64), nkeys - 1)
    key_bits = np.where(np.arange(nkeys) < nkeys // 2, 128, 256).astype(np.int32)
    offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    return RequestMix(sizes, modes.astype(np.int32), dirs, keys, key_bits, offsets)


def poisson_arrivals(seed: int, n: int, rate_per_s: float) -> np.ndarray:
    """Open-loop arrival times (seconds from 0) of a Poisson process."""
    u = uniform01(seed, STREAM_ARRIVAL, n)
    gaps = -np.log1p(-u) / rate_per_s
    return np.cumsum(gaps)


def mix_key_material(seed: int, mix: RequestMix) -> list[bytes]:
    """Raw key bytes per key index: XTS needs 2x key length, so 64 bytes are drawn
    per key and each mode takes the prefix it needs."""
    out = []
    for k, bits in enumerate(mix.key_bits):
        raw = bytes(seeded_bytes(seed, STREAM_KEY, 64 * (k + 1))[64 * k: 64 * (k + 1)])
        nb = int(bits) // 8
        if raw[:nb] == raw[nb:2 * nb]:
            raise ValueError("seeded XTS key halves collide")
        out.append(raw)
    return out


__all__ = [n for n in dir() if not n.startswith("_")]
