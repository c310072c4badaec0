"""Counter-based random numbers for the oracle: Philox4x32-10 and the
Gaussian directions z_k ~ N(0, I_n) of Sec. IV-B (Eq. random_directions).

TEST INFRASTRUCTURE ONLY, like the rest of oracle/.  The CUDA library draws
the same numbers on the device from its own implementation; the two share no
code and meet only through the published definition of the generator.

Philox4x32-10 (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as
easy as 1, 2, 3", SC 2011): a 128-bit counter c = (c0, c1, c2, c3) and a
64-bit key k = (k0, k1).  One round with multipliers M0 = 0xD2511F53 and
M1 = 0xCD9E8D57 maps
    c -> (hi(M1 c2) xor c1 xor k0, lo(M1 c2), hi(M0 c0) xor c3 xor k1, lo(M0 c0))
where hi/lo are the upper/lower 32 bits of the 64-bit product; the key is
bumped by (0x9E3779B9, 0xBB67AE85) between rounds; ten rounds.

Directions: pair g of the n x N_r row-major array (elements 2g, 2g+1) takes
the block at counter (g mod 2^32, g div 2^32, 0, 0) with key (seed mod 2^32,
seed div 2^32); words (x0, x1) and (x2, x3) give 53-bit uniforms
u = ((x_a >> 6) * 2^27 + (x_b >> 5) + 1/2) * 2^-53, and Box-Muller gives
r cos(2 pi u2), r sin(2 pi u2), r = sqrt(-2 ln u1).
"""
from __future__ import annotations

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(counter, key):
    """Philox4x32-10 of counters (array of shape (..., 4), uint32 values) under
    key (k0, k1); returns an array of the same shape (uint64 holding uint32)."""
    c = np.array(counter, dtype=np.uint64).reshape(-1, 4) & MASK
    k0, k1 = np.uint64(key[0] & MASK), np.uint64(key[1] & MASK)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(W0)) & np.uint64(MASK)
            k1 = (k1 + np.uint64(W1)) & np.uint64(MASK)
        p0 = np.uint64(M0) * c[:, 0]
        p1 = np.uint64(M1) * c[:, 2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & np.uint64(MASK)
        hi1, lo1 = p1 >> np.uint64(32), p1 & np.uint64(MASK)
        c = np.stack([hi1 ^ c[:, 1] ^ k0, lo1, hi0 ^ c[:, 3] ^ k1, lo0], axis=1)
    return c.reshape(np.shape(counter))


def philox_blocks(seed: int, counter0: int, count: int) -> np.ndarray:
    """Words of `count` consecutive blocks starting at counter0 (64-bit counter
    in (c0, c1)), as a flat uint32 array of 4 * count entries."""
    g = np.arange(counter0, counter0 + count, dtype=np.uint64)
    ctr = np.stack([g & np.uint64(MASK), g >> np.uint64(32), np.zeros_like(g), np.zeros_like(g)], axis=1)
    return philox4x32_10(ctr, (seed & MASK, (seed >> 32) & MASK)).astype(np.uint32).reshape(-1)


def _uniform53(a, b):
    m = (a.astype(np.uint64) >> np.uint64(6)) * np.uint64(1 << 27) + (b.astype(np.uint64) >> np.uint64(5))
    return (m.astype(np.float64) + 0.5) * 2.0 ** -53


def gaussian_directions(seed: int, n: int, n_r: int) -> np.ndarray:
    """Z (n x N_r, row-major float64) with z_k ~ N(0, I_n), column k = z_k."""
    count = n * n_r
    pairs = (count + 1) // 2
    w = philox_blocks(seed, 0, pairs).reshape(pairs, 4)
    u1 = _uniform53(w[:, 0], w[:, 1])
    u2 = _uniform53(w[:, 2], w[:, 3])
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * pairs)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:count].reshape(n, n_r)
