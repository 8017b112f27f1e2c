"""Philox4x32-10 counter-based generator, uniforms and Box-Muller normals.

The paper draws random numbers in Alg. 1 (initial prior draws, resampling),
Alg. 2 (proposal noise, component choice, the accept test) and the mixture fit,
but names no generator.  Both this oracle and the CUDA library use
Philox4x32-10 as defined by Salmon, Moraes, Dror and Shaw, "Parallel Random
Numbers: As Easy as 1, 2, 3" (SC'11): a 4-word counter, a 2-word key, ten
rounds of two 32x32->64 multiplies with the published multipliers, the key
bumped by the published Weyl constants between rounds.  Each side implements
it from that definition; nothing is shared.

Stream layout (a reading; the paper is silent):
  key     = (seed & 0xffffffff, seed >> 32)
  counter = (word-group index, particle index, step counter, purpose tag)
"""
import numpy as np

# Published constants (Salmon et al., SC'11, Philox4x32).
PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85

# Purpose tags (4th counter word).
INIT, COMP, NORMAL, ACCEPT, RESAMPLE, EMINIT, DATA, TRUTH, JITTER = 1, 2, 3, 4, 5, 6, 7, 8, 9

_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox rounds on counters (broadcastable uint32 arrays) with key (k0, k1).

    Returns four uint32 arrays.  One round: the products M0*c0 and M1*c2 are
    split into high and low halves; the new counter is
    (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)).
    """
    c0, c1, c2, c3 = np.broadcast_arrays(*(np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3)))
    c0, c1, c2, c3 = (c.copy() for c in (c0, c1, c2, c3))
    k0 = np.uint64(k0) & _MASK
    k1 = np.uint64(k1) & _MASK
    m0 = np.uint64(PHILOX_M0)
    m1 = np.uint64(PHILOX_M1)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(PHILOX_W0)) & _MASK
            k1 = (k1 + np.uint64(PHILOX_W1)) & _MASK
        p0 = m0 * c0          # < 2^64, exact in uint64
        p1 = m1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return tuple(c.astype(np.uint32) for c in (c0, c1, c2, c3))


def key_of(seed):
    seed = int(seed)
    return seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF


def u53(wa, wb):
    """53-bit integer from two 32-bit words: top 27 bits of wa, top 26 bits of wb."""
    wa = np.asarray(wa, dtype=np.uint64)
    wb = np.asarray(wb, dtype=np.uint64)
    return ((wa >> np.uint64(5)) << np.uint64(26)) | (wb >> np.uint64(6))


def uniform_open(wa, wb):
    """U = (u53 + 1/2) * 2^-53, strictly inside (0, 1); exact in binary64."""
    return (u53(wa, wb).astype(np.float64) + 0.5) * 2.0 ** -53


def uniforms(seed, c0, c1, c2, purpose):
    """One open-interval uniform per counter, from words 0 and 1."""
    k0, k1 = key_of(seed)
    w = philox4x32_10(c0, c1, c2, purpose, k0, k1)
    return uniform_open(w[0], w[1])


def normal_pairs(seed, npairs, c1, c2, purpose):
    """Box-Muller pairs: counter (m, c1, c2, purpose), m = 0..npairs-1, gives
    U1 from words (0, 1) and U2 from words (2, 3); R = sqrt(-2 log U1),
    z_{2m} = R cos(2 pi U2), z_{2m+1} = R sin(2 pi U2).

    Returns an array of 2*npairs normals; c1, c2 are scalars.
    """
    k0, k1 = key_of(seed)
    m = np.arange(npairs, dtype=np.uint64)
    w = philox4x32_10(m, c1, c2, purpose, k0, k1)
    u1 = uniform_open(w[0], w[1])
    u2 = uniform_open(w[2], w[3])
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * npairs)
    z[0::2] = r * np.cos(2.0 * np.pi * u2)
    z[1::2] = r * np.sin(2.0 * np.pi * u2)
    return z


def normals(seed, count, c1, c2, purpose):
    """count standard normals (count rounded up to pairs, then truncated)."""
    return normal_pairs(seed, (count + 1) // 2, c1, c2, purpose)[:count]


def word32(seed, c0, c1, c2, purpose, which=0):
    """A raw 32-bit word (for integer draws such as indices)."""
    k0, k1 = key_of(seed)
    return philox4x32_10(c0, c1, c2, purpose, k0, k1)[which]
