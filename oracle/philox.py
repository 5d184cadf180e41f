"""Counter-based random numbers for the oracle: Philox4x32-10 + Box-Muller.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package. The CUDA library implements the same generator independently from
the same published definition; the two share no code.

Definition followed: Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as
easy as 1, 2, 3" (SC'11), the Philox-4x32 bijection with 10 rounds:

    round(c, k):  (hi0, lo0) = mulhilo32(0xD2511F53, c0)
                  (hi1, lo1) = mulhilo32(0xCD9E8D57, c2)
                  c' = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
    key schedule: k0 += 0x9E3779B9, k1 += 0xBB67AE85 between rounds.

The paper (Alg. 1 and Alg. 2) only requires independent Gaussian draws; the
counter layout below is this library's own convention and is the one the
CUDA side uses, so that both sides see identical draws:

    key     = (seed & 0xffffffff, seed >> 32)
    counter = (word, t | purpose << 24, iteration & 0xffffffff, chain)

Each counter yields four 32-bit words. Word r becomes the uniform
u = ((r >> 9) + 0.5) * 2**-23, which lies in (0, 1) and is exactly
representable in both binary32 and binary64. Box-Muller turns the pairs
(r0, r1) and (r2, r3) into four standard normals; normal i of a
(chain, iteration, purpose, t) stream is component i % 4 of word i // 4.
"""
import numpy as np

PHILOX_M0 = 0xD2511F53
PHILOX_M1 = 0xCD9E8D57
PHILOX_W0 = 0x9E3779B9
PHILOX_W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

# stream purposes (the ``purpose`` field of the counter)
PURPOSE_AUX = 0        # u_t = x_t + sqrt(delta/2) * eps_t          (Alg. 2, first line)
PURPOSE_BACKWARD = 1   # noise of U_t in the backward sampler        (Appendix A.2.2)
PURPOSE_MH = 2         # the uniform of the Metropolis-Hastings test (Alg. 2, MRTH line)


def philox4x32_10(counter, key):
    """Philox4x32-10 on arrays.

    counter: uint array [..., 4]; key: uint array [..., 2] (broadcastable).
    Returns uint32 array [..., 4].
    """
    c = np.asarray(counter, dtype=np.uint64) & MASK32
    k = np.asarray(key, dtype=np.uint64) & MASK32
    c0, c1, c2, c3 = (c[..., i].copy() for i in range(4))
    k0 = np.broadcast_to(k[..., 0], c0.shape).copy()
    k1 = np.broadcast_to(k[..., 1], c0.shape).copy()
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = np.uint64(PHILOX_M0) * c0
        p1 = np.uint64(PHILOX_M1) * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return np.stack([c0, c1, c2, c3], axis=-1).astype(np.uint32)


def words_to_uniform(r):
    """uint32 -> uniform in (0,1): ((r >> 9) + 0.5) * 2^-23 (exact in fp32/fp64)."""
    r = np.asarray(r, dtype=np.uint64)
    return ((r >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23


def _counters(seed, chain, iteration, purpose, t, nwords):
    chain = np.asarray(chain, dtype=np.uint64)
    t = np.asarray(t, dtype=np.uint64)
    shape = np.broadcast_shapes(chain.shape, t.shape)
    chain = np.broadcast_to(chain, shape)
    t = np.broadcast_to(t, shape)
    w = np.arange(nwords, dtype=np.uint64)
    ctr = np.empty(shape + (nwords, 4), dtype=np.uint64)
    ctr[..., 0] = w
    ctr[..., 1] = ((t & np.uint64(0xFFFFFF)) | (np.uint64(purpose) << np.uint64(24)))[..., None]
    ctr[..., 2] = np.uint64(int(iteration) & MASK32)
    ctr[..., 3] = chain[..., None]
    key = np.array([int(seed) & MASK32, (int(seed) >> 32) & MASK32], dtype=np.uint64)
    return ctr, key


def normals(seed, chain, iteration, purpose, t, d):
    """Standard normals of the (chain, iteration, purpose, t) streams.

    chain and t broadcast against each other; returns float64 [..., d].
    """
    nwords = (d + 3) // 4
    ctr, key = _counters(seed, chain, iteration, purpose, t, nwords)
    r = philox4x32_10(ctr, key)                      # [..., nwords, 4]
    u = words_to_uniform(r)
    rad01 = np.sqrt(-2.0 * np.log(u[..., 0]))
    ang01 = 2.0 * np.pi * u[..., 1]
    rad23 = np.sqrt(-2.0 * np.log(u[..., 2]))
    ang23 = 2.0 * np.pi * u[..., 3]
    z = np.stack([rad01 * np.cos(ang01), rad01 * np.sin(ang01),
                  rad23 * np.cos(ang23), rad23 * np.sin(ang23)], axis=-1)
    z = z.reshape(z.shape[:-2] + (nwords * 4,))
    return z[..., :d]


def path_normals(seed, chain, iteration, purpose, T, d):
    """Normals for a whole path: float64 [T, d] (or [C, T, d] if chain is an array)."""
    chain = np.asarray(chain)
    t = np.arange(T)
    if chain.ndim == 0:
        return normals(seed, chain, iteration, purpose, t, d)
    return normals(seed, chain[:, None], iteration, purpose, t[None, :], d)


def mh_uniform(seed, chain, iteration):
    """The Metropolis-Hastings uniform of (chain, iteration): word 0 of t = 0."""
    ctr, key = _counters(seed, chain, iteration, PURPOSE_MH, 0, 1)
    r = philox4x32_10(ctr, key)
    return words_to_uniform(r[..., 0, 0])
