"""Random draws of the adaptive setup (oracle side).

The adaptive setup starts from randomly chosen vectors (paper: "a randomly
chosen initial error vector", Eq. relax). The oracle and the CUDA library each
implement the same counter-based generator from its published definition:
Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11; multipliers 0xD2511F53,
0xCD9E8D57, Weyl increments 0x9E3779B9, 0xBB67AE85) followed by Box-Muller.

Draw of level vector k on level l (0 = finest), complex dof index i:
    key     = (seed mod 2^32, seed >> 32)
    counter = (i mod 2^32, i >> 32, k, l)
    a = (w1 * 2^32 + w0) >> 11,  b = (w3 * 2^32 + w2) >> 11
    u1 = (a + 1) 2^-53 in (0, 1],  u2 = b 2^-53 in [0, 1)
    z  = sqrt(-2 ln u1) (cos 2 pi u2 + i sin 2 pi u2)
"""
from __future__ import annotations

import numpy as np

_MASK = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10 on uint32 values held in uint64 arrays."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3))
    k0 = np.uint64(int(k0) & 0xFFFFFFFF)
    k1 = np.uint64(int(k1) & 0xFFFFFFFF)
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return c0, c1, c2, c3


def gaussian_vector(n: int, seed: int, k: int, level: int) -> np.ndarray:
    """n complex Gaussians of setup vector k on ``level`` (see module docstring)."""
    i = np.arange(n, dtype=np.uint64)
    w0, w1, w2, w3 = philox4x32_10(i & _MASK, i >> np.uint64(32), np.full(n, k, dtype=np.uint64),
                                   np.full(n, level, dtype=np.uint64), seed & 0xFFFFFFFF, seed >> 32)
    a = ((w1 << np.uint64(32)) | w0) >> np.uint64(11)
    b = ((w3 << np.uint64(32)) | w2) >> np.uint64(11)
    u1 = (a.astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = b.astype(np.float64) * 2.0 ** -53
    rad = np.sqrt(-2.0 * np.log(u1))
    return rad * np.cos(2 * np.pi * u2) + 1j * rad * np.sin(2 * np.pi * u2)
