"""Philox4x32-10 counter-based random numbers (test infrastructure only).

Follows the published definition of Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3" (SC'11), Philox-4x32 with
ten rounds: two 32x32->64 multiplies per round with the multipliers
0xD2511F53 and 0xCD9E8D57, the key bumped by the Weyl constants
0x9E3779B9 and 0xBB67AE85 between rounds.

The paper under study does not name a generator.  The PQMC sweep reads it in
one fixed way, stated here and mirrored by the CUDA path from the same
published definition (the two share no code):

* key     = (seed & 0xffffffff, seed >> 32)
* counter = (site i, slice tau, sweep index, chain index)
* Metropolis uniform u = ((x0 << 21) | (x1 >> 11)) * 2**-53, in [0, 1)
* initial field s = +1 iff (x2 & 1) == 1, drawn with sweep index 0xffffffff
"""
import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF
INIT_SWEEP = 0xFFFFFFFF


def philox4x32_10(counter, key):
    """One Philox4x32-10 block: 4 counter words, 2 key words -> 4 words."""
    c0, c1, c2, c3 = (int(x) & MASK for x in counter)
    k0, k1 = (int(x) & MASK for x in key)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK
        hi1, lo1 = p1 >> 32, p1 & MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return (c0, c1, c2, c3)


def philox4x32_10_vec(c0, c1, c2, c3, k0, k1):
    """Vectorised form over numpy uint64 arrays holding 32-bit words."""
    c0 = np.asarray(c0, dtype=np.uint64) & MASK
    c1 = np.asarray(c1, dtype=np.uint64) & MASK
    c2 = np.asarray(c2, dtype=np.uint64) & MASK
    c3 = np.asarray(c3, dtype=np.uint64) & MASK
    k0 = np.uint64(k0 & MASK)
    k1 = np.uint64(k1 & MASK)
    m0 = np.uint64(M0)
    m1 = np.uint64(M1)
    mask = np.uint64(MASK)
    sh = np.uint64(32)
    for rnd in range(10):
        if rnd > 0:
            k0 = np.uint64((int(k0) + W0) & MASK)
            k1 = np.uint64((int(k1) + W1) & MASK)
        p0 = m0 * c0
        p1 = m1 * c2
        hi0, lo0 = p0 >> sh, p0 & mask
        hi1, lo1 = p1 >> sh, p1 & mask
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def seed_key(seed):
    seed = int(seed)
    return (seed & MASK, (seed >> 32) & MASK)


def uniform(seed, chain, sweep, tau, i):
    """Metropolis uniform for proposal (chain, sweep, tau, i)."""
    x0, x1, _, _ = philox4x32_10((i, tau, sweep, chain), seed_key(seed))
    return ((x0 << 21) | (x1 >> 11)) * 2.0 ** -53


def uniforms_slice(seed, chain, sweep, tau, n):
    """Uniforms for sites 0..n-1 of one slice (vectorised, same values)."""
    k0, k1 = seed_key(seed)
    i = np.arange(n, dtype=np.uint64)
    x0, x1, _, _ = philox4x32_10_vec(i, np.full(n, tau), np.full(n, sweep),
                                     np.full(n, chain), k0, k1)
    return ((x0 << np.uint64(21)) | (x1 >> np.uint64(11))).astype(np.float64) * 2.0 ** -53


def initial_fields(seed, chain, n_slices, n_sites):
    """Initial Ising fields s[tau][i] in {-1,+1} (int8)."""
    k0, k1 = seed_key(seed)
    tau, i = np.meshgrid(np.arange(n_slices, dtype=np.uint64),
                         np.arange(n_sites, dtype=np.uint64), indexing="ij")
    _, _, x2, _ = philox4x32_10_vec(i, tau, np.full(i.shape, INIT_SWEEP),
                                    np.full(i.shape, chain), k0, k1)
    return np.where((x2 & np.uint64(1)) == 1, 1, -1).astype(np.int8)
