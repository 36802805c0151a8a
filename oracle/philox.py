"""Counter-based Philox4x32-10 generator and its Box-Muller normals (oracle side).

TEST INFRASTRUCTURE ONLY.  Written from the published definition of Philox in
Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11):
a 4x32-bit counter and a 2x32-bit key; each of the 10 rounds multiplies counter words
0 and 2 by two fixed odd constants, keeps the high and low halves of the 64-bit
products, and mixes the high halves with words 1 and 3 and with the round key; the
key is bumped by the two Weyl constants between rounds.

The paper draws its complex-Langevin noise on the device (CURAND, Sec. "CUDA
implementation"); a counter-based generator lets the oracle reproduce the device
stream exactly.  Stream layout shared by both sides (defined by this project):
key = (seed mod 2^32, seed >> 32); counter = (point // 4, field, step, instance); one
call yields four uint32 words (x0, x1, x2, x3) which Box-Muller turns into the normals
of points 4p .. 4p+3 as r1 cos t1, r1 sin t1, r2 cos t2, r2 sin t2 with
u = (x + 1/2) 2^-32, r = sqrt(-2 ln u_even), t = 2 pi u_odd.
"""
from __future__ import annotations

import numpy as np

_MUL0 = np.uint64(0xD2511F53)
_MUL1 = np.uint64(0xCD9E8D57)
_WEYL0 = 0x9E3779B9
_WEYL1 = 0xBB67AE85
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(counters, key):
    """Philox4x32 with 10 rounds.

    counters: uint32 array of shape (..., 4); key: pair of ints.  Returns uint32 array
    of the same shape."""
    c = np.asarray(counters, dtype=np.uint64)
    c0, c1, c2, c3 = (c[..., i].copy() for i in range(4))
    k0 = int(key[0]) & 0xFFFFFFFF
    k1 = int(key[1]) & 0xFFFFFFFF
    for _ in range(10):
        p0 = _MUL0 * c0          # < 2^64: both factors < 2^32
        p1 = _MUL1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK32
        n0 = hi1 ^ c1 ^ np.uint64(k0)
        n2 = hi0 ^ c3 ^ np.uint64(k1)
        c0, c1, c2, c3 = n0, lo1, n2, lo0
        k0 = (k0 + _WEYL0) & 0xFFFFFFFF
        k1 = (k1 + _WEYL1) & 0xFFFFFFFF
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def _uniform_open(x):
    """uint32 -> double in (0, 1): (x + 1/2) * 2^-32."""
    return (x.astype(np.float64) + 0.5) * (1.0 / 4294967296.0)


def philox_normals(seed: int, instance: int, step: int, field: int, M: int) -> np.ndarray:
    """Standard normals for grid points 0..M-1 of one (instance, step, field) stream."""
    nblk = (M + 3) // 4
    ctr = np.zeros((nblk, 4), dtype=np.uint64)
    ctr[:, 0] = np.arange(nblk, dtype=np.uint64)
    ctr[:, 1] = field
    ctr[:, 2] = step & 0xFFFFFFFF
    ctr[:, 3] = instance & 0xFFFFFFFF
    x = philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))
    u0, u1, u2, u3 = (_uniform_open(x[:, i]) for i in range(4))
    r1 = np.sqrt(-2.0 * np.log(u0))
    r2 = np.sqrt(-2.0 * np.log(u2))
    t1 = 2.0 * np.pi * u1
    t2 = 2.0 * np.pi * u3
    z = np.stack([r1 * np.cos(t1), r1 * np.sin(t1), r2 * np.cos(t2), r2 * np.sin(t2)], axis=-1)
    return z.reshape(-1)[:M]
