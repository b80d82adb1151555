"""Philox4x32-10 counter-based generator, written from its published definition.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC'11: one round maps counter (c0, c1, c2, c3) and key (k0, k1) to
  (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
with M0 = 0xD2511F53, M1 = 0xCD9E8D57; between rounds the key is bumped by the
Weyl constants (0x9E3779B9, 0xBB67AE85).  Ten rounds.

Vectorised over numpy uint64 arrays holding 32-bit values.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)
S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    c = [np.asarray(x, dtype=np.uint64) & MASK for x in (c0, c1, c2, c3)]
    k0 = np.asarray(k0, dtype=np.uint64) & MASK
    k1 = np.asarray(k1, dtype=np.uint64) & MASK
    for rnd in range(10):
        if rnd:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        c = [((p1 >> S32) ^ c[1] ^ k0) & MASK, p1 & MASK, ((p0 >> S32) ^ c[3] ^ k1) & MASK, p0 & MASK]
    return c


def u53(a, b):
    """Uniform double in [0, 1) from two 32-bit words: (a >> 11, b) as a 53-bit integer times 2^-53."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    return (((a >> np.uint64(11)) << S32) | b).astype(np.float64) * (2.0 ** -53)


def index_below(a, b, n):
    """floor(u * n / 2^64) with u = a * 2^32 + b: an exact integer in [0, n) (n < 2^31)."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    n = np.asarray(n, dtype=np.uint64)
    return ((a * n + ((b * n) >> S32)) >> S32).astype(np.int64)


def normal_pair(a, b, c, d):
    """Two standard normals by the Box-Muller transform of u1 = u53(a,b), u2 = u53(c,d)."""
    u1 = u53(a, b)
    u2 = u53(c, d)
    rad = np.sqrt(-2.0 * np.log(1.0 - u1))
    return rad * np.cos(2.0 * np.pi * u2), rad * np.sin(2.0 * np.pi * u2)
