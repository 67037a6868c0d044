"""Philox4x64-10 counter-based generator and the complex Gaussian vectors
SIM-M's multiplicity step draws (Sec. 3.4: "k random vectors").

TEST INFRASTRUCTURE ONLY (part of the oracle).  Written from the published
definition (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11): two 64×64→128-bit multiplies per round with multipliers
0xD2E7470EE14C6C93 and 0xCA5A826395121157, Weyl key increments
0x9E3779B97F4A7C15 and 0xBB67AE8584CAA73B, 10 rounds.

Element e of random vector v for seed s: counter (e, v, 0, 0), key
(s, 0x53494D4D).  Words 0 and 1 give two uniforms u = (x >> 11) * 2^-53;
Box–Muller gives re + i im = sqrt(-2 ln(1-u0)) e^{2πi u1} / sqrt(2).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2E7470EE14C6C93)
M1 = np.uint64(0xCA5A826395121157)
W0 = np.uint64(0x9E3779B97F4A7C15)
W1 = np.uint64(0xBB67AE8584CAA73B)
KEY1 = 0x53494D4D
_LO32 = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(a, b):
    """Full 128-bit product of uint64 arrays, as (hi, lo), from 32-bit halves."""
    a_lo, a_hi = a & _LO32, a >> _S32
    b_lo, b_hi = b & _LO32, b >> _S32
    ll = a_lo * b_lo
    lh = a_lo * b_hi
    hl = a_hi * b_lo
    hh = a_hi * b_hi
    mid = (ll >> _S32) + (lh & _LO32) + (hl & _LO32)
    lo = (ll & _LO32) | ((mid & _LO32) << _S32)
    hi = hh + (lh >> _S32) + (hl >> _S32) + (mid >> _S32)
    return hi, lo


def philox4x64(counter, key, rounds: int = 10):
    """Philox4x64-R on arrays: counter is a 4-tuple of uint64 arrays, key a 2-tuple."""
    x0, x1, x2, x3 = (np.asarray(c, dtype=np.uint64) for c in counter)
    k0, k1 = (np.asarray(k, dtype=np.uint64) for k in key)
    with np.errstate(over="ignore"):
        for _ in range(rounds):
            hi0, lo0 = _mulhilo(M0, x0)
            hi1, lo1 = _mulhilo(M1, x2)
            x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
            k0 = k0 + W0
            k1 = k1 + W1
    return x0, x1, x2, x3


def random_vectors(seed: int, n: int, k: int, first: int = 0) -> np.ndarray:
    """n × k complex128 matrix; column v is random vector (first + v)."""
    e = np.repeat(np.arange(n, dtype=np.uint64)[:, None], k, axis=1)
    v = np.repeat(np.arange(first, first + k, dtype=np.uint64)[None, :], n, axis=0)
    zero = np.zeros_like(e)
    x0, x1, _, _ = philox4x64((e, v, zero, zero), (np.uint64(seed), np.uint64(KEY1)))
    u0 = (x0 >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    u1 = (x1 >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    r = np.sqrt(-2.0 * np.log1p(-u0))
    th = 2.0 * np.pi * u1
    return (r * np.cos(th) + 1j * (r * np.sin(th))) * 0.70710678118654752440
