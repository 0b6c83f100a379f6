"""Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11), written from the published definition: ten rounds of two 32x32->64
bit multiplications with key bumps by the Weyl constants between rounds.

Used by the oracle wherever the method draws random numbers: entries of the initial MPS
and the uniforms of the sequential sampler.  Pinned by the published known-answer
vectors (tests/golden/philox4x32_10_kat.txt).
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK = np.uint64(0xFFFFFFFF)

STREAM_INIT = 1      # counter word 3 for initial-MPS entries
STREAM_SAMPLE = 2    # counter word 3 for sampler uniforms
STREAM_TRUNC = 3     # counter word 3 for the start vectors of the warm-started truncation


def philox4x32_10(ctr, key):
    """ctr: uint array [..., 4], key: uint array [..., 2] (broadcastable).  Returns
    uint64 array [..., 4] holding the four 32-bit output words."""
    c = np.asarray(ctr, dtype=np.uint64) & MASK
    k = np.asarray(key, dtype=np.uint64) & MASK
    c0, c1, c2, c3 = c[..., 0], c[..., 1], c[..., 2], c[..., 3]
    k0, k1 = k[..., 0], k[..., 1]
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0            # < 2**64, exact in uint64
        p1 = M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK, lo1, (hi0 ^ c3 ^ k1) & MASK, lo0
    return np.stack([c0, c1, c2, c3], axis=-1)


def key_of(seed: int):
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return np.array([seed & 0xFFFFFFFF, seed >> 32], dtype=np.uint64)


def uniform53(x_hi, x_lo):
    """Double in [0, 1) from two 32-bit words: 32 bits of x_hi then the top 21 of x_lo."""
    v = (np.asarray(x_hi, dtype=np.uint64) << np.uint64(21)) | (np.asarray(x_lo, dtype=np.uint64) >> np.uint64(11))
    return v.astype(np.float64) * (2.0 ** -53)


def counters(index, word2: int, stream: int):
    index = np.asarray(index, dtype=np.uint64)
    ctr = np.zeros(index.shape + (4,), dtype=np.uint64)
    ctr[..., 0] = index & MASK
    ctr[..., 1] = index >> np.uint64(32)
    ctr[..., 2] = np.uint64(word2)
    ctr[..., 3] = np.uint64(stream)
    return ctr


def complex_normals(seed: int, site: int, count: int, stream: int = STREAM_INIT):
    """count complex numbers z = (g1 + i g2)/sqrt(2), g ~ N(0,1) by Box-Muller, from the
    given stream of (seed, site): entry j uses counter (j, site, stream)."""
    out = philox4x32_10(counters(np.arange(count, dtype=np.uint64), site, stream), key_of(seed))
    u1 = uniform53(out[..., 0], out[..., 1])
    u2 = uniform53(out[..., 2], out[..., 3])
    rad = np.sqrt(-2.0 * np.log1p(-u1))
    ang = 2.0 * np.pi * u2
    return (rad * np.cos(ang) + 1j * rad * np.sin(ang)) / np.sqrt(2.0)


def sample_uniforms(seed: int, sample_index, site: int):
    """Uniform double of the SAMPLE stream for (seed, sample, site)."""
    out = philox4x32_10(counters(sample_index, site, STREAM_SAMPLE), key_of(seed))
    return uniform53(out[..., 0], out[..., 1])
