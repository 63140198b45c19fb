"""Counter-based random numbers for same-draw parity.

Test infrastructure (see the package docstring).  Written from the published
definition of Philox4x32 with 10 rounds (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11): per round two 32x32
-> 64-bit products of counter words 0 and 2 with the multipliers
0xD2511F53 / 0xCD9E8D57, the output words (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1,
lo0), and a Weyl bump of the key by 0x9E3779B9 / 0xBB67AE85 between rounds.

Stream layout shared with the CUDA path (an interface, not code):
key = (seed & 0xffffffff, seed >> 32); counter = (j, sample, stream, 0).
Normal number 2j and 2j+1 of (sample, stream) come from counter j: words
(0,1) and (2,3) form two 53-bit uniforms u1, u2 in (0, 1), and Box-Muller
(1958) gives r cos(2 pi u2), r sin(2 pi u2) with r = sqrt(-2 log u1).
Rademacher value 4j + w is 1 - 2 (word_w & 1).  Streams: 0 = prior rows,
1 = observation rows, 2 = probes.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)

STREAM_PRIOR = 0
STREAM_OBS = 1
STREAM_PROBE = 2


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10.  Inputs are integer arrays (or scalars) of
    32-bit values; returns four uint64 arrays holding 32-bit words."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & MASK for v in (c0, c1, c2, c3))
    k0 = np.uint64(k0) & MASK
    k1 = np.uint64(k1) & MASK
    for r in range(10):
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK, lo1, (hi0 ^ c3 ^ k1) & MASK, lo0
        if r < 9:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
    return c0, c1, c2, c3


def _key(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def _u53(a, b):
    """Uniform in (0, 1) from two 32-bit words: ((a >> 5) 2^26 + (b >> 6) + 1/2) 2^-53."""
    hi = (a >> np.uint64(5)).astype(np.float64)
    lo = (b >> np.uint64(6)).astype(np.float64)
    return (hi * 67108864.0 + lo + 0.5) / 9007199254740992.0


def normals(seed: int, stream: int, sample: int, n: int) -> np.ndarray:
    """n standard normals of one (sample, stream)."""
    k0, k1 = _key(seed)
    npair = (n + 1) // 2
    j = np.arange(npair, dtype=np.uint64)
    x0, x1, x2, x3 = philox4x32_10(j, np.uint64(sample), np.uint64(stream), np.uint64(0), k0, k1)
    u1 = _u53(x0, x1)
    u2 = _u53(x2, x3)
    r = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * npair)
    out[0::2] = r * np.cos(2.0 * np.pi * u2)
    out[1::2] = r * np.sin(2.0 * np.pi * u2)
    return out[:n]


def rademacher(seed: int, sample: int, n: int) -> np.ndarray:
    k0, k1 = _key(seed)
    nq = (n + 3) // 4
    j = np.arange(nq, dtype=np.uint64)
    words = philox4x32_10(j, np.uint64(sample), np.uint64(STREAM_PROBE), np.uint64(0), k0, k1)
    out = np.empty(4 * nq)
    for w in range(4):
        out[w::4] = 1.0 - 2.0 * (words[w] & np.uint64(1)).astype(np.float64)
    return out[:n]
