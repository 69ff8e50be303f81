"""Philox4x32-10 counter-based generator and Box-Muller normals, written from their published
definitions (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3",
SC 2011; Box and Muller, 1958). The device draws the randomized-range-finder test matrix of
eq. rrf from the same definition, so both sides see the same numbers without storing them.

Test infrastructure only (see the package docstring).

Entry (l, j) of the p x r_hat test matrix Omega: counter (l mod 2^32, l div 2^32, j, 0), key
(seed mod 2^32, seed div 2^32); of the four output words x0..x3, u1 = (x0 + 1/2) 2^-32 and
u2 = (x1 + 1/2) 2^-32 give Omega[l, j] = sqrt(-2 ln u1) cos(2 pi u2).
"""

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57   # round multipliers
W0, W1 = 0x9E3779B9, 0xBB67AE85   # key increments (Weyl sequence)
MASK = 0xFFFFFFFF


def _mulhilo(a, b):
    prod = a.astype(np.uint64) * np.uint64(b)
    return (prod >> np.uint64(32)).astype(np.uint64), (prod & np.uint64(MASK)).astype(np.uint64)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten rounds of Philox4x32 on counters (arrays of uint) with key (k0, k1): each round maps
    (c0, c1, c2, c3) to (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)), and the
    key advances by (W0, W1) between rounds. Returns four uint64 arrays holding 32-bit words."""
    c = [np.asarray(x, dtype=np.uint64) & np.uint64(MASK) for x in (c0, c1, c2, c3)]
    k0 = np.uint64(k0 & MASK)
    k1 = np.uint64(k1 & MASK)
    for rnd in range(10):
        if rnd > 0:
            k0 = np.uint64((int(k0) + W0) & MASK)
            k1 = np.uint64((int(k1) + W1) & MASK)
        hi0, lo0 = _mulhilo(c[0], M0)
        hi1, lo1 = _mulhilo(c[2], M1)
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return c


def gaussian_test_matrix(p, r_hat, seed):
    """Omega (p x r_hat, FP64) of eq. rrf from Philox4x32-10 + Box-Muller, as described above."""
    l = np.arange(p, dtype=np.uint64)[:, None] * np.ones((1, r_hat), dtype=np.uint64)
    j = np.ones((p, 1), dtype=np.uint64) * np.arange(r_hat, dtype=np.uint64)[None, :]
    x = philox4x32_10(l & np.uint64(MASK), l >> np.uint64(32), j, np.zeros_like(j),
                      seed & MASK, (seed >> 32) & MASK)
    u1 = (x[0].astype(np.float64) + 0.5) * 2.0 ** -32
    u2 = (x[1].astype(np.float64) + 0.5) * 2.0 ** -32
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
