"""Counter-based Gaussian test matrices for the oracle (FP64, numpy).

The paper draws the test matrix Omega_n from a Gaussian distribution
(Section 3.1, the paragraph before Eq. (sampleMatrix)); Algorithm 1 step (5)
writes ``rand`` and the remark after Algorithm 1 allows uniform entries.  The
reading taken here is Gaussian.  Because the CUDA path regenerates Omega in
registers instead of storing it, both sides implement one counter-based
generator from its published definition:

* Philox4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
  easy as 1, 2, 3", SC'11): a 4x32-bit counter, a 2x32-bit key, ten rounds of
  two 32x32->64 multiplications with the constants 0xD2511F53 / 0xCD9E8D57,
  and a Weyl key schedule with increments 0x9E3779B9 / 0xBB67AE85.
* Box-Muller: z0 = sqrt(-2 ln u1) cos(2 pi u2), z1 = sqrt(-2 ln u1) sin(2 pi u2).

Stream layout (shared definition, written independently on each side):
  key     = (seed mod 2^32, seed div 2^32)
  counter = (g mod 2^32, g div 2^32, stream, purpose)
where ``g`` is the pair index (element index e of a row-major rows x cols
matrix, g = e div 2, element parity picks z0/z1), ``stream`` is the 1-based
mode number n and ``purpose`` is PURPOSE_SKETCH for Omega_n or
PURPOSE_ALS_INIT for the seeded ALS initial factors.

FP64 uniforms take 53 bits from two words: u = ((w0 >> 5) * 2^26 + (w1 >> 6)) * 2^-53,
u1 = 1 - u_a in (0, 1] from words (x0, x1) and u2 = u_b in [0, 1) from (x2, x3).

The reduced-precision ("f32") stream used by the tensor-core sweeps takes four
normals per counter: for k in {0, 1}, u1 = ((x_{2k} >> 8) + 1) * 2^-24,
u2 = (x_{2k+1} >> 8) * 2^-24, z_{2k}, z_{2k+1} by Box-Muller; element e maps
to counter g = e div 4 and slot e mod 4.
"""

import numpy as np

PURPOSE_SKETCH = 0
PURPOSE_ALS_INIT = 1

_MASK = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on arrays of 32-bit words (held in uint64).

    Each round: (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
    c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0); then the key advances by
    the Weyl increments.  Returns four uint64 arrays of 32-bit values.
    """
    c0 = np.asarray(c0, dtype=np.uint64) & _MASK
    c1 = np.asarray(c1, dtype=np.uint64) & _MASK
    c2 = np.asarray(c2, dtype=np.uint64) & _MASK
    c3 = np.asarray(c3, dtype=np.uint64) & _MASK
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & _MASK, lo1, (hi0 ^ c3 ^ k1) & _MASK, lo0
        k0 = (k0 + _W0) & _MASK
        k1 = (k1 + _W1) & _MASK
    return c0, c1, c2, c3


def _words(seed, stream, purpose, g):
    g = np.asarray(g, dtype=np.uint64)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return philox4x32_10(g & _MASK, g >> np.uint64(32),
                         np.full_like(g, stream), np.full_like(g, purpose),
                         seed & 0xFFFFFFFF, seed >> 32)


def _u53(hi, lo):
    return ((hi >> np.uint64(5)).astype(np.float64) * 67108864.0
            + (lo >> np.uint64(6)).astype(np.float64)) * (1.0 / 9007199254740992.0)


def normals_f64(seed, stream, purpose, count):
    """The first ``count`` FP64 normals of one stream (element e -> pair e // 2)."""
    npairs = (int(count) + 1) // 2
    x0, x1, x2, x3 = _words(seed, stream, purpose, np.arange(npairs, dtype=np.uint64))
    u1 = 1.0 - _u53(x0, x1)
    u2 = _u53(x2, x3)
    r = np.sqrt(-2.0 * np.log(u1))
    th = 2.0 * np.pi * u2
    z = np.empty(2 * npairs, dtype=np.float64)
    z[0::2] = r * np.cos(th)
    z[1::2] = r * np.sin(th)
    return z[:count]


def normals_f32_stream(seed, stream, purpose, count):
    """The reduced-precision stream's values, evaluated in FP64 (element e -> counter e // 4)."""
    nq = (int(count) + 3) // 4
    x = _words(seed, stream, purpose, np.arange(nq, dtype=np.uint64))
    z = np.empty(4 * nq, dtype=np.float64)
    for k in range(2):
        u1 = ((x[2 * k] >> np.uint64(8)).astype(np.float64) + 1.0) * 2.0 ** -24
        u2 = (x[2 * k + 1] >> np.uint64(8)).astype(np.float64) * 2.0 ** -24
        r = np.sqrt(-2.0 * np.log(u1))
        z[2 * k::4] = r * np.cos(2.0 * np.pi * u2)
        z[2 * k + 1::4] = r * np.sin(2.0 * np.pi * u2)
    return z[:count]


def gaussian_matrix(seed, stream, purpose, rows, cols):
    """rows x cols FP64 matrix of standard normals, element (j, c) at e = j*cols + c."""
    return normals_f64(seed, stream, purpose, rows * cols).reshape(rows, cols)
