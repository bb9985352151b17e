"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11).

One call maps a 128-bit counter and a 64-bit key to 128 random bits through ten
rounds of two 32x32->64 multiplies and a Feistel-like xor/permute, with a Weyl
key schedule. Written from the published definition; checked against the
known-answer vectors published with the Random123 library.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint32(0x9E3779B9)
W1 = np.uint32(0xBB67AE85)
_MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Apply Philox4x32 with 10 rounds. Counters are uint32 arrays (broadcastable),
    keys uint32 scalars or arrays. Returns four uint32 arrays."""
    c0 = np.asarray(c0, dtype=np.uint32)
    c1 = np.asarray(c1, dtype=np.uint32)
    c2 = np.asarray(c2, dtype=np.uint32)
    c3 = np.asarray(c3, dtype=np.uint32)
    k0 = np.asarray(k0, dtype=np.uint32)
    k1 = np.asarray(k1, dtype=np.uint32)
    c0, c1, c2, c3 = np.broadcast_arrays(c0, c1, c2, c3)
    with np.errstate(over="ignore"):
        for r in range(10):
            if r > 0:
                k0 = (k0 + W0).astype(np.uint32)
                k1 = (k1 + W1).astype(np.uint32)
            p0 = M0 * c0.astype(np.uint64)
            p1 = M1 * c2.astype(np.uint64)
            hi0 = (p0 >> np.uint64(32)).astype(np.uint32)
            lo0 = (p0 & _MASK32).astype(np.uint32)
            hi1 = (p1 >> np.uint64(32)).astype(np.uint32)
            lo1 = (p1 & _MASK32).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def uniform01(seed, stream, start, count, indices=None):
    """Doubles in the open interval (0, 1) for indices start..start+count-1 (or the given
    index array).

    Counter = (index low 32 bits, index high 32 bits, stream, 0), key = (seed, 0x524F5821).
    The first two output words form a 53-bit mantissa: u = (a>>5 * 2^26 + b>>6 + 0.5) / 2^53.
    """
    if indices is not None:
        idx = np.asarray(indices, dtype=np.uint64)
    else:
        idx = np.arange(start, start + count, dtype=np.uint64)
    lo = (idx & _MASK32).astype(np.uint32)
    hi = (idx >> np.uint64(32)).astype(np.uint32)
    x0, x1, _, _ = philox4x32_10(lo, hi, np.uint32(stream), np.uint32(0),
                                 np.uint32(seed), np.uint32(0x524F5821))
    a = (x0 >> np.uint32(5)).astype(np.float64)
    b = (x1 >> np.uint32(6)).astype(np.float64)
    return (a * 67108864.0 + b + 0.5) / 9007199254740992.0
