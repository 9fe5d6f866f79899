"""Counter-based Gaussian draws for the compression matrices (FP64 CPU oracle).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg, never by the product path.  It shares no code
with the CUDA library, which implements the same published generator on its
own.

The Gaussian compression matrix Omega (Sec. 3.1, i.i.d. N(0, 1) entries) and
the fresh per-block draws of repeated sampling (Sec. 3.4) can be produced
from a seed by a counter-based generator, so that a draw is a pure function
of (seed, substream, position).  The generator is Philox4x32-10 (Salmon,
Moraes, Dror and Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11),
followed by the Box-Muller transform (Box and Muller, 1958):

* Philox4x32 round on counter (c0, c1, c2, c3) with key (k0, k1):
  (hi0, lo0) = 0xD2511F53 * c0 and (hi1, lo1) = 0xCD9E8D57 * c2 as 64-bit
  products split into 32-bit halves; the new counter is
  (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0).  Ten rounds; between rounds the
  key advances by the Weyl constants (0x9E3779B9, 0xBB67AE85) mod 2^32.
* Stream layout (a convention of this library, not of the paper): the key is
  the 64-bit seed (k0 = low word, k1 = high word); entry q = i + j * l of the
  l x m matrix (column-major position, independent of the leading dimension)
  belongs to the Philox call with counter (t mod 2^32, t >> 32, s mod 2^32,
  s >> 32), t = q // 2, s = the substream.  The four output words x0..x3
  give two uniforms u_1 = ((x0 x1 as a 64-bit word >> 12) + 1/2) 2^-52 and
  u_2 likewise from x2 x3, both strictly inside (0, 1) and exact in FP64.
* Box-Muller: r = sqrt(-2 ln u_1); entry 2t is r cos(2 pi u_2) and entry
  2t + 1 is r sin(2 pi u_2).
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """Philox4x32-10 of an (N, 4) array of 32-bit counters under a 2-word key."""
    c = np.asarray(ctr, dtype=np.uint64).reshape(-1, 4) & MASK32
    c0, c1, c2, c3 = (c[:, i].copy() for i in range(4))
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for _ in range(10):
        p0 = M0 * c0                      # < 2^64: exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0)
        k0 = (k0 + W0) & 0xFFFFFFFF
        k1 = (k1 + W1) & 0xFFFFFFFF
    return np.stack([c0, c1, c2, c3], axis=1).astype(np.uint32)


def uniforms(words):
    """Two uniforms in (0, 1) per Philox output: (x0:x1 >> 12 + 1/2) 2^-52, (x2:x3 ...)."""
    w = np.asarray(words, dtype=np.uint64)
    a = ((w[:, 0] << np.uint64(32)) | w[:, 1]) >> np.uint64(12)
    b = ((w[:, 2] << np.uint64(32)) | w[:, 3]) >> np.uint64(12)
    scale = 2.0 ** -52
    return (a.astype(np.float64) + 0.5) * scale, (b.astype(np.float64) + 0.5) * scale


def gaussian(seed, l, m, substream=0):
    """The l x m Gaussian matrix of (seed, substream), FP64 (Sec. 3.1's Omega)."""
    total = l * m
    npairs = (total + 1) // 2
    t = np.arange(npairs, dtype=np.uint64)
    s = int(substream)
    ctr = np.stack([t & MASK32, t >> np.uint64(32),
                    np.full(npairs, s & 0xFFFFFFFF, dtype=np.uint64),
                    np.full(npairs, (s >> 32) & 0xFFFFFFFF, dtype=np.uint64)], axis=1)
    seed = int(seed)
    u1, u2 = uniforms(philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)))
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * npairs)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z[:total].reshape(m, l).T.copy()


def resampler(seed):
    """Draws for repeated sampling: block J's fresh l x m_t Gaussian is substream J."""
    return lambda J, l, mt: gaussian(seed, l, mt, substream=J)
