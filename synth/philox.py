"""Philox4x32-10 counter-based generator (Salmon et al., SC'11) in vectorised numpy.

Definition used (the published one): a 128-bit counter (c0, c1, c2, c3) and a
64-bit key (k0, k1) go through ten rounds.  One round multiplies c0 and c2 by
the constants 0xD2511F53 and 0xCD9E8D57 into 64-bit products (hi, lo) and
returns (hi(c2*M1) ^ c1 ^ k0, lo(c2*M1), hi(c0*M0) ^ c3 ^ k1, lo(c0*M0)).
Between rounds the key is bumped by the Weyl constants (0x9E3779B9,
0xBB67AE85).  The CUDA library implements the same definition independently.

Stream layout (shared convention, stated here once):
  key      = (seed & 0xffffffff, seed >> 32)
  normals  : element with flat index f uses counter (j & 0xffffffff, j >> 32,
             stream, 0) with j = f // 2; the four words give two 52-bit
             uniforms u1, u2 and Box-Muller gives sqrt(-2 ln u1) * cos(2 pi u2)
             for even f and sqrt(-2 ln u1) * sin(2 pi u2) for odd f.
  uniforms : element i uses counter (j & 0xffffffff, j >> 32, stream, 1) with
             j = i // 2; words (0, 1) give element 2j and words (2, 3) give
             element 2j + 1.
  uniform52(a, b) = ((a >> 6) * 2**26 + (b >> 6) + 0.5) * 2**-52, in (0, 1):
             52 random bits plus a half-step offset, every value exactly
             representable (so 0 and 1 never occur).
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = np.uint64(0xFFFFFFFF)

STREAM_X0 = 1
STREAM_BDIAG = 2
STREAM_COEF = 3
STREAM_POTENTIAL = 4
STREAM_OMEGA = 5
STREAM_GRAD = 6


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on arrays of 32-bit counter words (any shape).

    Returns four uint64 arrays holding the 32-bit output words.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & MASK32
    c1 = np.asarray(c1, dtype=np.uint64) & MASK32
    c2 = np.asarray(c2, dtype=np.uint64) & MASK32
    c3 = np.asarray(c3, dtype=np.uint64) & MASK32
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & 0xFFFFFFFF
            k1 = (k1 + W1) & 0xFFFFFFFF
        p0 = M0 * c0          # < 2**64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                          hi0 ^ c3 ^ np.uint64(k1), lo0)
    return c0, c1, c2, c3


def uniform52(a, b):
    """Map two 32-bit words to a double in (0, 1): 52 random bits + 1/2 ulp offset."""
    a = np.asarray(a, dtype=np.uint64)
    b = np.asarray(b, dtype=np.uint64)
    m = (a >> np.uint64(6)) * np.uint64(1 << 26) + (b >> np.uint64(6))
    return (m.astype(np.float64) + 0.5) * (2.0 ** -52)


def _key(seed):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return seed & 0xFFFFFFFF, seed >> 32


def normal_flat(seed, stream, start, count):
    """Standard normals for flat indices start .. start+count-1 of a stream."""
    k0, k1 = _key(seed)
    out = np.empty(count, dtype=np.float64)
    chunk = 1 << 22
    for s in range(0, count, chunk):
        f = np.arange(start + s, start + min(count, s + chunk), dtype=np.uint64)
        j = f >> np.uint64(1)
        x0, x1, x2, x3 = philox4x32_10(j & MASK32, j >> np.uint64(32),
                                        np.uint64(stream), np.uint64(0), k0, k1)
        u1 = uniform52(x0, x1)
        u2 = uniform52(x2, x3)
        r = np.sqrt(-2.0 * np.log(u1))
        ang = 2.0 * np.pi * u2
        odd = (f & np.uint64(1)).astype(bool)
        out[s:s + len(f)] = np.where(odd, r * np.sin(ang), r * np.cos(ang))
    return out


def normal_block(seed, stream, rows, cols, row0=0):
    """Row-major rows x cols block of N(0, 1) samples; row r is global row row0 + r."""
    return normal_flat(seed, stream, row0 * cols, rows * cols).reshape(rows, cols)


def uniform_block(seed, stream, count, lo=0.0, hi=1.0):
    """count uniforms on (lo, hi) from the given stream."""
    k0, k1 = _key(seed)
    out = np.empty(count, dtype=np.float64)
    chunk = 1 << 22
    for s in range(0, count, chunk):
        i = np.arange(s, min(count, s + chunk), dtype=np.uint64)
        j = i >> np.uint64(1)
        x0, x1, x2, x3 = philox4x32_10(j & MASK32, j >> np.uint64(32),
                                        np.uint64(stream), np.uint64(1), k0, k1)
        odd = (i & np.uint64(1)).astype(bool)
        u = np.where(odd, uniform52(x2, x3), uniform52(x0, x1))
        out[s:s + len(i)] = lo + (hi - lo) * u
    return out
