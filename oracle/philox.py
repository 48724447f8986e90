"""Counter-based Gaussian test matrices for the oracle.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Philox4x32-10 is written from its published definition (J. Salmon, M. Moraes,
R. Dror, D. Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11,
Sec. 5): a 4-word counter and 2-word key; each of the 10 rounds multiplies
words 0 and 2 by two fixed odd constants, recombines the high and low halves
with the other words and the round key, and the key is bumped by two Weyl
constants between rounds.

The Gaussian transform is Box and Muller (1958): two uniforms u1, u2 in (0,1)
give sqrt(-2 ln u1) cos(2 pi u2) and sqrt(-2 ln u1) sin(2 pi u2).

Omega of mode k (Alg. 3 step 3) is an n x b matrix whose entry (i, c) is the
(c mod 4)-th Gaussian produced from counter (i mod 2^32, i >> 32, c // 4, k)
under key (seed mod 2^32, seed >> 32), with uniforms
u(x) = ((x >> 9) + 1/2) * 2^-23, exactly representable in binary32.
Entries depend only on (seed, k, i, c), so the columns for oversampling p are
a prefix of those for p + 1.  This file evaluates the transform in float64.
"""
import numpy as np

_MUL0 = 0xD2511F53
_MUL1 = 0xCD9E8D57
_WEYL0 = 0x9E3779B9
_WEYL1 = 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32_10(counter, key):
    """Philox4x32 with 10 rounds.

    counter: array-like of shape (..., 4) of uint32 words; key: (2,) words.
    Returns uint32 array of shape (..., 4).
    """
    ctr = np.asarray(counter, dtype=np.uint64)
    c0, c1, c2, c3 = (ctr[..., i].copy() for i in range(4))
    k0 = np.uint64(int(key[0]) & _MASK)
    k1 = np.uint64(int(key[1]) & _MASK)
    m0 = np.uint64(_MUL0)
    m1 = np.uint64(_MUL1)
    mask = np.uint64(_MASK)
    s32 = np.uint64(32)
    for _ in range(10):
        p0 = m0 * c0                    # exact: both factors < 2^32
        p1 = m1 * c2
        hi0, lo0 = p0 >> s32, p0 & mask
        hi1, lo1 = p1 >> s32, p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + np.uint64(_WEYL0)) & mask
        k1 = (k1 + np.uint64(_WEYL1)) & mask
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def _uniform(x):
    """(0,1) uniform from a 32-bit word, exactly representable in binary32."""
    return ((x.astype(np.uint64) >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def omega_from_seed(seed, k, n, b, row_start=0, row_stop=None):
    """Rows [row_start, row_stop) of the n x b Gaussian Omega of mode k."""
    seed = int(seed)
    if row_stop is None:
        row_stop = n
    rows = np.arange(row_start, row_stop, dtype=np.uint64)
    groups = (b + 3) // 4
    out = np.empty((rows.size, groups * 4), dtype=np.float64)
    key = (seed & _MASK, (seed >> 32) & _MASK)
    for g in range(groups):
        ctr = np.empty((rows.size, 4), dtype=np.uint64)
        ctr[:, 0] = rows & np.uint64(_MASK)
        ctr[:, 1] = rows >> np.uint64(32)
        ctr[:, 2] = g
        ctr[:, 3] = k
        x = philox4x32_10(ctr, key)
        for pair in range(2):
            u1 = _uniform(x[:, 2 * pair])
            u2 = _uniform(x[:, 2 * pair + 1])
            rad = np.sqrt(-2.0 * np.log(u1))
            ang = 2.0 * np.pi * u2
            out[:, 4 * g + 2 * pair] = rad * np.cos(ang)
            out[:, 4 * g + 2 * pair + 1] = rad * np.sin(ang)
    return out[:, :b]
