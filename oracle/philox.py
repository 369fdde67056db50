"""Oracle (test infrastructure only): the Gaussian test matrix Omega of Alg. 4, step 3.

The paper only says ``Omega = randn(n, l)`` (Alg. 1 step 2, Alg. 4 step 3). This
module fixes one reproducible reading of that draw so that the oracle and the
CUDA library can be compared on the same Omega:

* integers: Philox4x32-10, the counter-based generator of Salmon, Moraes, Dror
  and Shaw, "Parallel random numbers: as easy as 1, 2, 3" (SC'11). A 128-bit
  counter (four 32-bit words) and a 64-bit key (two words) are mapped through
  ten rounds; each round multiplies counter words 0 and 2 by two fixed odd
  constants, keeps both halves of the 64-bit products and xors the high halves
  with counter words 1 and 3 and the key; the key is advanced by two Weyl
  increments between rounds.
* uniforms: u = (x + 1/2) * 2^-32 for each 32-bit word x, computed in FP64
  (exact: 33 significant bits), so 0 < u < 1.
* normals: the Box-Muller transform (Box & Muller, 1958) on pairs of uniforms:
  r = sqrt(-2 ln u0), z0 = r cos(2 pi u1), z1 = r sin(2 pi u1).
* layout: Omega[j, 4q + t] (t = 0..3) comes from the counter
  (j mod 2^32, j div 2^32, q, stream 0) under the key (seed mod 2^32,
  seed div 2^32); words (x0, x1) give z0, z1 and words (x2, x3) give z2, z3.
  Columns at or beyond l are discarded, so Omega does not depend on padding.

Everything here is plain numpy on uint64 words and float64 values.
"""
import numpy as np

MASK32 = np.uint64(0xFFFFFFFF)
# Philox4x32 round multipliers and key increments as published by Salmon et al.
PHILOX_M0 = np.uint64(0xD2511F53)
PHILOX_M1 = np.uint64(0xCD9E8D57)
PHILOX_W0 = np.uint64(0x9E3779B9)
PHILOX_W1 = np.uint64(0xBB67AE85)
PHILOX_ROUNDS = 10

STREAM_OMEGA = 0


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32-10 on arrays of counters; returns the four output words (uint32).

    c0..c3 are broadcastable integer arrays (counter words), k0/k1 the key words.
    """
    x = [np.asarray(c, dtype=np.uint64) & MASK32 for c in (c0, c1, c2, c3)]
    x0, x1, x2, x3 = np.broadcast_arrays(*x)
    key0 = np.uint64(k0) & MASK32
    key1 = np.uint64(k1) & MASK32
    for r in range(PHILOX_ROUNDS):
        if r > 0:
            key0 = (key0 + PHILOX_W0) & MASK32
            key1 = (key1 + PHILOX_W1) & MASK32
        prod0 = PHILOX_M0 * x0          # < 2^64: exact in uint64
        prod1 = PHILOX_M1 * x2
        hi0, lo0 = prod0 >> np.uint64(32), prod0 & MASK32
        hi1, lo1 = prod1 >> np.uint64(32), prod1 & MASK32
        x0, x1, x2, x3 = hi1 ^ x1 ^ key0, lo1, hi0 ^ x3 ^ key1, lo0
    return tuple(w.astype(np.uint32) for w in (x0, x1, x2, x3))


def seed_key(seed):
    """Split a 64-bit seed into the two Philox key words (low word first)."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def omega_words(n, l, seed, stream=STREAM_OMEGA):
    """Raw Philox words behind Omega: uint32 array of shape (n, 4*ceil(l/4))."""
    q_count = (l + 3) // 4
    j = np.arange(n, dtype=np.uint64)[:, None]
    q = np.arange(q_count, dtype=np.uint64)[None, :]
    k0, k1 = seed_key(seed)
    w = philox4x32_10(j & MASK32, j >> np.uint64(32), q, np.uint64(stream), k0, k1)
    out = np.empty((n, q_count, 4), dtype=np.uint32)
    for t in range(4):
        out[:, :, t] = w[t]
    return out.reshape(n, 4 * q_count)


def uniforms(words):
    """u = (x + 1/2) 2^-32 in FP64, strictly inside (0, 1)."""
    return (words.astype(np.float64) + 0.5) * (2.0 ** -32)


def box_muller(u0, u1):
    """Box-Muller pair of standard normals from two independent uniforms."""
    r = np.sqrt(-2.0 * np.log(u0))
    theta = 2.0 * np.pi * u1
    return r * np.cos(theta), r * np.sin(theta)


def omega(n, l, seed, stream=STREAM_OMEGA):
    """The n x l Gaussian test matrix Omega (FP64), Alg. 4 step 3."""
    u = uniforms(omega_words(n, l, seed, stream))
    z = np.empty_like(u)
    z[:, 0::4], z[:, 1::4] = box_muller(u[:, 0::4], u[:, 1::4])
    z[:, 2::4], z[:, 3::4] = box_muller(u[:, 2::4], u[:, 3::4])
    return z[:, :l].copy()
