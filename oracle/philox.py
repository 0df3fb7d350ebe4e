"""Counter-based Gaussian probes for the randomized sketches (oracle).

Algorithm 1 and Algorithm 2 draw an n x r matrix Omega of standard normal
numbers.  For complex matrices the oracle reads "standard normal" as complex
standard normal: real and imaginary parts iid N(0, 1/2), so E|w|^2 = 1.

The numbers come from Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel
random numbers: as easy as 1, 2, 3", SC'11), written here from that
definition, so that the CUDA path can draw the identical stream on its own:

  round:  (c0, c1, c2, c3) -> (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2),
                               hi(M0 c0) ^ c3 ^ k1, lo(M0 c0))
  key schedule between rounds: k0 += W0, k1 += W1 (mod 2^32)
  M0 = 0xD2511F53, M1 = 0xCD9E8D57, W0 = 0x9E3779B9, W1 = 0xBB67AE85.

Entry (i, j) of a probe block with 64-bit seed s and stream words (w2, w3):
  counter = (i >> 1, j, w2, w3), key = (s mod 2^32, s >> 32);
  (x0, x1) of the output for even i, (x2, x3) for odd i;
  u1 = (xa + 1) 2^-32 in (0, 1],  u2 = xb 2^-32 in [0, 1);
  Omega_ij = sqrt(-ln u1) (cos 2 pi u2 + i sin 2 pi u2)        (Box-Muller).

Stream words name the sketch: tag in bits 28-31 of w2 (1: H-matrix build,
2: global sketch of the simple preconditioner, 3: recompression inside the
H-matrix inversion), op in bits 24-27, (level, node) of the inversion call in
bits 16-23 / 0-15, and w3 = (block level << 16) | block node.
"""
from __future__ import annotations

import numpy as np

M0, M1 = 0xD2511F53, 0xCD9E8D57
W0, W1 = 0x9E3779B9, 0xBB67AE85
MASK = 0xFFFFFFFF

TAG_BUILD, TAG_GLOBAL, TAG_RECOMPRESS = 1, 2, 3


def stream_words(tag: int, op: int = 0, lvl: int = 0, node: int = 0,
                 blvl: int = 0, bnode: int = 0):
    w2 = ((tag & 0xF) << 28) | ((op & 0xF) << 24) | ((lvl & 0xFF) << 16) | (node & 0xFFFF)
    w3 = ((blvl & 0xFFFF) << 16) | (bnode & 0xFFFF)
    return w2, w3


def philox4x32_10(ctr, key):
    """Philox4x32-10 on uint64 arrays holding 32-bit words (vectorised).

    ``ctr`` is a tuple of four arrays, ``key`` a tuple of two ints."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & MASK for c in ctr)
    k0, k1 = np.uint64(key[0] & MASK), np.uint64(key[1] & MASK)
    m0, m1 = np.uint64(M0), np.uint64(M1)
    mask, sh = np.uint64(MASK), np.uint64(32)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + np.uint64(W0)) & mask
            k1 = (k1 + np.uint64(W1)) & mask
        p0 = m0 * c0           # < 2^64: exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> sh, p0 & mask
        hi1, lo1 = p1 >> sh, p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def gaussian(rows: int, cols: int, seed: int, w2: int, w3: int) -> np.ndarray:
    """The rows x cols complex Gaussian probe block defined above."""
    i = np.arange(rows, dtype=np.uint64)[:, None] * np.ones((1, cols), dtype=np.uint64)
    j = np.ones((rows, 1), dtype=np.uint64) * np.arange(cols, dtype=np.uint64)[None, :]
    key = (seed & MASK, (seed >> 32) & MASK)
    x0, x1, x2, x3 = philox4x32_10((i >> np.uint64(1), j, np.full_like(i, w2), np.full_like(i, w3)), key)
    odd = (i & np.uint64(1)).astype(bool)
    xa = np.where(odd, x2, x0).astype(np.float64)
    xb = np.where(odd, x3, x1).astype(np.float64)
    u1 = (xa + 1.0) * 2.0 ** -32
    u2 = xb * 2.0 ** -32
    rho = np.sqrt(-np.log(u1))
    return rho * np.cos(2 * np.pi * u2) + 1j * rho * np.sin(2 * np.pi * u2)
