"""Philox-4x32-10 counter-based generator and the Gaussian white noise of the ICs.

Test infrastructure only.  Written from the published definition (Salmon,
Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11):
ten rounds of

    (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0,  lo(M1 c2),  hi(M0 c0) ^ c3 ^ k1,  lo(M0 c0))

with M0 = 0xD2511F53, M1 = 0xCD9E8D57 and the key bumped by the Weyl
constants (0x9E3779B9, 0xBB67AE85) between rounds.

White noise of the initial conditions (this build's recipe; the paper gives none):
the lattice point with linear index idx = (z N + y) N + x uses counter
(idx mod 2^32, idx div 2^32, 0, 0) and key (seed mod 2^32, seed div 2^32); the
first two output words give u_i = (w_i + 1/2)/2^32 and
g = sqrt(-2 ln u1) cos(2 pi u2) in double precision (Box-Muller).

Pins (tests/test_oracle_basics.py): the published known-answer vectors of
Philox-4x32-10; moments of the normal deviates.
"""
from __future__ import annotations

import numpy as np

M0, M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
W0, W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)
S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox-4x32-10; all arguments uint32-valued arrays (held as uint64)."""
    c0, c1, c2, c3 = (np.asarray(v, dtype=np.uint64) & MASK for v in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK
    k1 = np.asarray(k1, dtype=np.uint64) & MASK
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0          # < 2^64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> S32, p0 & MASK
        hi1, lo1 = p1 >> S32, p1 & MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def white_noise(N: int, seed: int) -> np.ndarray:
    """Unit-variance Gaussian white noise on an N^3 lattice, indexed [z][y][x], float64."""
    idx = np.arange(N**3, dtype=np.uint64)
    seed = int(seed)
    r0, r1, _, _ = philox4x32_10(idx & MASK, idx >> S32, 0, 0,
                                 np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF))
    u1 = (r0.astype(np.float64) + 0.5) / 4294967296.0
    u2 = (r1.astype(np.float64) + 0.5) / 4294967296.0
    g = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return g.reshape(N, N, N)
