"""Philox4x32-10, written from its published definition (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11, Sec. 3.2 and Table 2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

One Philox round maps the counter (c0, c1, c2, c3) under key (k0, k1) to
    (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
and the key is bumped by the Weyl constants (W0, W1) between rounds; ten rounds.

The uniform used everywhere in this project is the 53-bit double
    u = ((x0 >> 5) * 2**26 + (x1 >> 6)) * 2**-53   in [0, 1)
built from the first two output words (the "res53" construction).

Counter layout (the method's random draws; key = the realization's 64-bit seed):
    bond b            : (b, 0, 0, PURPOSE_BOND)
    spin at site i    : (i, step, chain, PURPOSE_SPIN)
    accept at a step  : (0, step, chain, PURPOSE_ACCEPT)
"""
import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK32 = 0xFFFFFFFF

PURPOSE_BOND = 0
PURPOSE_SPIN = 1
PURPOSE_ACCEPT = 2


def philox4x32_10(ctr, key):
    """Philox4x32-10 on broadcastable integer arrays.

    ctr: sequence of 4 arrays (counter words), key: sequence of 2 arrays.
    Returns a tuple of 4 uint64 arrays holding the 32-bit output words.
    """
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & np.uint64(MASK32) for x in ctr)
    k0, k1 = (np.asarray(x, dtype=np.uint64) & np.uint64(MASK32) for x in key)
    m32 = np.uint64(MASK32)
    sh = np.uint64(32)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + np.uint64(W0)) & m32
            k1 = (k1 + np.uint64(W1)) & m32
        p0 = np.uint64(M0) * c0          # < 2**64: exact in uint64
        p1 = np.uint64(M1) * c2
        hi0, lo0 = p0 >> sh, p0 & m32
        hi1, lo1 = p1 >> sh, p1 & m32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & m32, lo1, (hi0 ^ c3 ^ k1) & m32, lo0
    return c0, c1, c2, c3


def seed_key(seed):
    """Split a 64-bit seed into the two 32-bit key words (low word first)."""
    seed = np.asarray(seed, dtype=np.uint64)
    return seed & np.uint64(MASK32), seed >> np.uint64(32)


def u53(x0, x1):
    """53-bit uniform double in [0, 1) from two 32-bit words."""
    a = (np.asarray(x0, dtype=np.uint64) >> np.uint64(5)).astype(np.float64)
    b = (np.asarray(x1, dtype=np.uint64) >> np.uint64(6)).astype(np.float64)
    return (a * 67108864.0 + b) * (1.0 / 9007199254740992.0)


def uniform(seed, c0, c1, c2, purpose):
    """The project's uniform for counter (c0, c1, c2, purpose) under ``seed``."""
    k0, k1 = seed_key(seed)
    x0, x1, _, _ = philox4x32_10((c0, c1, c2, purpose), (k0, k1))
    return u53(x0, x1)
