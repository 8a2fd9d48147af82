"""Seeded synthetic inputs shared by the library's tests, benchmark and oracle checks.

This module holds no stencil arithmetic: it only draws numbers. The paper's
benchmarks (Section 4.1, Table 1) run on synthetic grids; the values are
not given, so inputs are drawn from a counter-based SplitMix64 stream:

    z_i   = splitmix64_mix(seed + (i + 1) * 0x9E3779B97F4A7C15)   (mod 2**64)
    U_i   = (z_i >> 11) * 2**-53                                  in [0, 1)

splitmix64_mix is Steele, Lea and Flood's SplitMix64 finaliser (OOPSLA
2014): xor-shift 30, multiply 0xBF58476D1CE4E5B9, xor-shift 27, multiply
0x94D049BB133111EB, xor-shift 31. Being counter based, element i of a
stream does not depend on how the stream is chunked.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO_M53 = float(2.0 ** -53)

#: Seed base for the workload recipes (arbitrary, fixed).
SEED_BASE = 2010048680


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Raw 64-bit outputs i = start .. start+count-1 of the stream `seed`."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def uniform(seed: int, count: int, start: int = 0, chunk: int = 1 << 24) -> np.ndarray:
    """count doubles uniform in [0, 1) (53-bit), elements start.. of stream seed."""
    out = np.empty(count, dtype=np.float64)
    for a in range(0, count, chunk):
        n = min(chunk, count - a)
        out[a:a + n] = (splitmix64(seed, start + a, n) >> np.uint64(11)).astype(np.float64) * _TWO_M53
    return out


def grid(seed: int, ext) -> np.ndarray:
    """A C-order float64 grid of shape ext with uniform [0, 1) entries."""
    ext = tuple(int(e) for e in ext)
    n = int(np.prod(ext)) if ext else 0
    return uniform(seed, n).reshape(ext)


def dyadic_grid(seed: int, ext, bits: int) -> np.ndarray:
    """Grid of k-bit dyadic rationals m / 2**bits, m uniform in [0, 2**bits)."""
    ext = tuple(int(e) for e in ext)
    n = int(np.prod(ext)) if ext else 0
    m = splitmix64(seed, 0, n) >> np.uint64(64 - bits)
    return (m.astype(np.float64) * float(2.0 ** -bits)).reshape(ext)


def normalized_weights(seed: int, k: int) -> np.ndarray:
    """K positive weights summing to (about) 1, in canonical offset order.

    r_i = 1 - U_i lies in (0, 1]; w_i = r_i / (r_0 + r_1 + ... + r_{K-1}),
    the sum taken left to right in float64. The rounded weights need not
    sum to exactly 1.
    """
    r = 1.0 - uniform(seed, k)
    s = 0.0
    for v in r:
        s = s + float(v)
    return np.array([float(v) / s for v in r], dtype=np.float64)


def normalized_field(seed: int, k: int, ext) -> np.ndarray:
    """Per-point weights for a variable-coefficient stencil: shape (k,) + ext, canonical term order.

    At every point p, r_q(p) = 1 - U lies in (0, 1] (U drawn term-major: all
    points of term 0, then term 1, ...) and f_q(p) = r_q(p) / (r_0(p) + ...
    + r_{k-1}(p)), the sum taken left to right in float64: positive weights
    summing to about 1 at each point, so repeated steps stay bounded.
    """
    ext = tuple(int(e) for e in ext)
    n = int(np.prod(ext)) if ext else 0
    r = (1.0 - uniform(seed, k * n)).reshape((k, n))
    s = np.zeros(n)
    for q in range(k):
        s = s + r[q]
    return (r / s).reshape((k,) + ext)


def cells(seed: int, ext, density: float = 0.5) -> np.ndarray:
    """A 0/1 uint8 grid: cell = 1 where U < density (U uniform [0, 1), SplitMix64 in C order)."""
    ext = tuple(int(e) for e in ext)
    n = int(np.prod(ext)) if ext else 0
    return (uniform(seed, n) < density).astype(np.uint8).reshape(ext)


def sequence(seed: int, n: int, sigma: int = 4) -> np.ndarray:
    """A uint8 sequence of n symbols drawn uniformly from {0, .., sigma - 1} (SplitMix64 modulo sigma)."""
    return (splitmix64(seed, 0, int(n)) % np.uint64(sigma)).astype(np.uint8)


def _i64(v: int) -> int:
    """A 64-bit pattern as a signed int64 value (two's complement)."""
    v &= 0xFFFFFFFFFFFFFFFF
    return v - (1 << 64) if v >= (1 << 63) else v


def grid_into(out, seed: int, chunk: int = 1 << 22):
    """Fill a float64 torch tensor (any device, contiguous) with the same values as grid(seed, out.shape).

    The same SplitMix64 stream, evaluated in torch int64 arithmetic (additions and products wrap
    modulo 2**64; a logical right shift is an arithmetic shift with the sign-extended bits masked
    off), a chunk of elements at a time so that temporaries stay small.
    """
    import torch
    flat = out.view(-1)
    n = flat.numel()
    g, m1, m2, s = _i64(0x9E3779B97F4A7C15), _i64(0xBF58476D1CE4E5B9), _i64(0x94D049BB133111EB), _i64(seed)

    def srl(x, k):
        return (x >> k) & ((1 << (64 - k)) - 1)

    for a in range(0, n, chunk):
        b = min(n, a + chunk)
        z = torch.arange(a + 1, b + 1, dtype=torch.int64, device=flat.device) * g + s
        z = z ^ srl(z, 30)
        z = z * m1
        z = z ^ srl(z, 27)
        z = z * m2
        z = z ^ srl(z, 31)
        flat[a:b] = srl(z, 11).to(torch.float64) * _TWO_M53
    return out

