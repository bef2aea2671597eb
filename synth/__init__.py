"""Seeded synthetic inputs for dedispersion tests and benchmarks.

This module holds no dedispersion arithmetic: it draws samples, packs them
into the time-major filterbank layout, and writes a boxcar along a delay row
that the caller supplies.  Both the CUDA path's tests and the oracle's tests
take their inputs from here; neither side imports the other.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: draw i of stream s under seed k is splitmix64(key(k, s) + i).

Layout written by ``pack``: row t holds channels 0..nchans-1; for nbits < 8
channel c sits at bits [(c*nbits) mod 8, +nbits) of byte (c*nbits)//8 of the
row, least significant bits first.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied to uint64 counters (wrapping)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def stream_key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        k = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * _GOLDEN ^ np.uint64(stream)
    return splitmix64(np.array([k], dtype=np.uint64))[0]


def draws(seed: int, stream: int, n: int, start: int = 0) -> np.ndarray:
    """n uint64 draws of (seed, stream) starting at counter ``start``."""
    key = stream_key(seed, stream)
    with np.errstate(over="ignore"):
        ctr = np.arange(start, start + n, dtype=np.uint64) + key
    return splitmix64(ctr)


def random_bytes(seed: int, stream: int, n: int) -> np.ndarray:
    """n uniformly distributed bytes (little-endian bytes of the draws)."""
    d = draws(seed, stream, (n + 7) // 8)
    return d.view(np.uint8)[:n].copy()


def uniform_samples(seed, stream, rows, nchans, nbits) -> np.ndarray:
    """uint8 [rows][nchans], each uniform on [0, 2**nbits)."""
    raw = random_bytes(seed, stream, rows * nchans)
    return (raw & np.uint8((1 << nbits) - 1)).reshape(rows, nchans)


def uniform_packed(seed, stream, rows, nchans, nbits) -> np.ndarray:
    """Packed rows whose nbits-wide fields are uniform: the bytes themselves
    are uniform, so this is random bytes (bits past the last channel zeroed)."""
    rb = (nchans * nbits + 7) // 8
    out = random_bytes(seed, stream, rows * rb).reshape(rows, rb)
    spare = rb * 8 - nchans * nbits
    if spare:
        out[:, -1] &= np.uint8((1 << (8 - spare)) - 1)
    return out


def _normal_from_draws(d: np.ndarray) -> np.ndarray:
    """Box-Muller on the two 32-bit halves of each draw: one N(0,1) each."""
    u1 = ((d >> np.uint64(32)).astype(np.float64) + 1.0) / 4294967296.0
    u2 = (d & np.uint64(0xFFFFFFFF)).astype(np.float64) / 4294967296.0
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def normal_u8(seed, stream, rows, nchans, mean=128.0, sd=16.0) -> np.ndarray:
    """uint8 [rows][nchans] = clip(floor(mean + sd*N(0,1) + 0.5), 0, 255)."""
    out = np.empty(rows * nchans, dtype=np.uint8)
    step = 1 << 24
    for s in range(0, rows * nchans, step):
        n = min(step, rows * nchans - s)
        z = _normal_from_draws(draws(seed, stream, n, start=s))
        out[s:s + n] = np.clip(np.floor(mean + sd * z + 0.5), 0, 255).astype(np.uint8)
    return out.reshape(rows, nchans)


def normal_f32(seed, stream, rows, nchans) -> np.ndarray:
    """float32 [rows][nchans] ~ N(0,1)."""
    out = np.empty(rows * nchans, dtype=np.float32)
    step = 1 << 24
    for s in range(0, rows * nchans, step):
        n = min(step, rows * nchans - s)
        out[s:s + n] = _normal_from_draws(draws(seed, stream, n, start=s))
    return out.reshape(rows, nchans)


def row_bytes(nchans: int, nbits: int) -> int:
    return (nchans * nbits + 7) // 8


def pack(samples: np.ndarray, nbits: int) -> np.ndarray:
    """uint8 [rows][nchans] samples -> packed uint8 [rows][row_bytes]."""
    s = np.ascontiguousarray(samples, dtype=np.uint8)
    rows, nchans = s.shape
    if nbits == 8:
        return s.copy()
    per = 8 // nbits
    pad = (-nchans) % per
    if pad:
        s = np.concatenate([s, np.zeros((rows, pad), np.uint8)], axis=1)
    s = s.reshape(rows, -1, per).astype(np.uint16)
    out = np.zeros(s.shape[:2], dtype=np.uint16)
    for k in range(per):
        out |= (s[:, :, k] & ((1 << nbits) - 1)) << (k * nbits)
    return out.astype(np.uint8)


def unpack(packed: np.ndarray, nbits: int, nchans: int) -> np.ndarray:
    """Inverse of ``pack``."""
    p = np.ascontiguousarray(packed, dtype=np.uint8)
    if nbits == 8:
        return p[:, :nchans].copy()
    per = 8 // nbits
    parts = [(p >> (k * nbits)) & ((1 << nbits) - 1) for k in range(per)]
    return np.stack(parts, axis=2).reshape(p.shape[0], -1)[:, :nchans].copy()


def inject_boxcar(samples: np.ndarray, delay_row, t0: int, width: int,
                  amp=None, value=None, maxval=255) -> np.ndarray:
    """Write a boxcar of ``width`` samples starting at t0 + delay_row[c] in
    every channel c of an unpacked [rows][nchans] array: add ``amp``
    (clipped at ``maxval``) or overwrite with ``value``.  Returns a copy."""
    out = np.array(samples, copy=True)
    delay_row = np.asarray(delay_row, dtype=np.int64)
    nchans = out.shape[1]
    for k in range(width):
        rows = t0 + delay_row + k
        ok = (rows >= 0) & (rows < out.shape[0])
        cols = np.arange(nchans)[ok]
        rr = rows[ok]
        if value is not None:
            out[rr, cols] = value
        else:
            v = out[rr, cols].astype(np.int64) + int(amp)
            out[rr, cols] = np.clip(v, 0, maxval).astype(out.dtype)
    return out


def inject_boxcar_packed(packed: np.ndarray, nbits: int, nchans: int, delay_row,
                         t0: int, width: int, value: int) -> np.ndarray:
    """``inject_boxcar`` with an overwrite value, directly on packed rows."""
    out = np.array(packed, copy=True)
    delay_row = np.asarray(delay_row, dtype=np.int64)
    chans = np.arange(nchans)
    byte = (chans * nbits) // 8
    shift = ((chans * nbits) % 8).astype(np.uint8)
    fmask = np.uint8((1 << nbits) - 1) if nbits < 8 else np.uint8(0xFF)
    for k in range(width):
        rows = t0 + delay_row + k
        ok = (rows >= 0) & (rows < out.shape[0])
        for r, b, s in zip(rows[ok], byte[ok], shift[ok]):
            cur = out[r, b]
            out[r, b] = (cur & ~np.uint8(fmask << s)) | np.uint8((value & fmask) << s)
    return out
