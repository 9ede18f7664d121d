"""Philox4x32-10 and the Gaussian white noise drawn from it (oracle side).

The paper does not say how its Gaussian field is drawn (Sec. sec_numerical,
"Gaussian Initial Conditions").  The reading used by both implementations:
white noise g(x) ~ N(0, 1) per lattice cell from the counter-based generator
Philox4x32 with 10 rounds, as published by Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11), followed by a
Box-Muller transform in FP64.

Counter / key assignment (the published generator is a pure function of both):
  key     = (seed & 0xffffffff, seed >> 32)
  counter = (cell, stream, 0, 0), cell = (i0 * N + i1) * N + i2 the row-major
            linear index of the lattice cell, stream = 0 for the noise field.
Box-Muller on the four output words (r0, r1, r2, r3):
  a  = ((r0 << 32) | r1) >> 11,  u1 = (a + 1) * 2**-53   in (0, 1]
  b  = ((r2 << 32) | r3) >> 11,  u2 = b * 2**-53         in [0, 1)
  g  = sqrt(-2 ln u1) * cos(2 pi u2)

Test infrastructure only (see the package docstring).
"""
import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def _mulhilo(a, b):
    """32x32 -> 64-bit product split into (hi, lo) words (uint64 arrays)."""
    p = a * b  # both < 2**32, the product fits in uint64
    return p >> _S32, p & _MASK


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds.

    ctr : tuple of four uint32-valued arrays (broadcastable), key : two words.
    Returns four uint64 arrays holding the 32-bit output words.

    One round (SC'11, Sec. 3): with multipliers M0, M1,
      (hi0, lo0) = M0 * c0 ;  (hi1, lo1) = M1 * c2
      c <- (hi1 ^ c1 ^ k0,  lo1,  hi0 ^ c3 ^ k1,  lo0)
    and the key is advanced by the Weyl constants (W0, W1) between rounds.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in ctr)
    k0 = np.uint64(int(key[0]) & 0xFFFFFFFF)
    k1 = np.uint64(int(key[1]) & 0xFFFFFFFF)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        hi0, lo0 = _mulhilo(_M0, c0)
        hi1, lo1 = _mulhilo(_M1, c2)
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def white_noise(N, seed, stream=0):
    """Real N^3 array (row-major [i0][i1][i2]) of N(0,1) draws, FP64."""
    cell = np.arange(N ** 3, dtype=np.uint64)
    zero = np.zeros_like(cell)
    seed = int(seed)
    r0, r1, r2, r3 = philox4x32_10(
        (cell, zero + np.uint64(stream), zero, zero),
        (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))
    a = ((r0 << _S32) | r1) >> np.uint64(11)
    b = ((r2 << _S32) | r3) >> np.uint64(11)
    u1 = (a.astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = b.astype(np.float64) * 2.0 ** -53
    g = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return g.reshape(N, N, N)
