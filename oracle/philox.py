"""Philox4x32-10 counter-based generator (test infrastructure only, see oracle/pc_engine.py).

Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3"
(SC'11): ten rounds of two 32x32 -> 64-bit products with the published
multipliers and Weyl key increments. The CUDA code implements the same
definition; draws that both sides must agree on (lattice vacancies, the visiting
order of position batches) are words of this generator.
"""
from __future__ import annotations

import numpy as np

_M0, _M1 = 0xD2511F53, 0xCD9E8D57
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32_10(counter, key):
    """counter: (..., 4) uint32-valued array; key: (2,) or (..., 2). Returns (..., 4) uint64 words < 2^32."""
    c = np.array(counter, dtype=np.uint64) & _MASK
    k = np.broadcast_to(np.array(key, dtype=np.uint64) & _MASK, c.shape[:-1] + (2,)).copy()
    c0, c1, c2, c3 = (c[..., i].copy() for i in range(4))
    k0, k1 = k[..., 0].copy(), k[..., 1].copy()
    for _ in range(10):
        p0 = np.uint64(_M0) * c0          # < 2^64: exact in uint64
        p1 = np.uint64(_M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(_MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(_MASK)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + np.uint64(_W0)) & np.uint64(_MASK)
        k1 = (k1 + np.uint64(_W1)) & np.uint64(_MASK)
    return np.stack([c0, c1, c2, c3], axis=-1)


def key_words(key64: int):
    return (key64 & _MASK, (key64 >> 32) & _MASK)


def permutation(n: int, key64: int, stream: int, t: int) -> np.ndarray:
    """Fisher-Yates shuffle of 0..n-1: for i = n-1 .. 1, j = (w (i + 1)) >> 32 with w the first
    word of Philox4x32-10((i, t, stream, 5), key); swap a[i], a[j]."""
    a = np.arange(n, dtype=np.int64)
    if n < 2:
        return a
    i = np.arange(n - 1, 0, -1, dtype=np.int64)
    ctr = np.stack([i, np.full_like(i, t & _MASK), np.full_like(i, stream), np.full_like(i, 5)], axis=-1)
    w = philox4x32_10(ctr.astype(np.uint64), key_words(key64))[:, 0]
    for ii, wi in zip(i, w):
        j = int((int(wi) * (int(ii) + 1)) >> 32)
        a[ii], a[j] = a[j], a[ii]
    return a
