"""Philox4x64-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as
1, 2, 3", SC'11), written from the published definition with Python integers.

The random spectrum permutation of Section 2.2 (Eq. 5-8) needs an odd scaling
sigma (invertible mod N, N a power of two) and a shift.  One (sigma, a) pair is drawn
per (signal, iteration m): all rounds of one multiscale location share sigma
(Section 3.2), and the per-level offsets follow from a (see ``plan``).

Pinned by: numpy's ``Philox`` bit generator (an independent Philox4x64-10), which
increments its 256-bit counter before producing each block.
"""

MASK64 = (1 << 64) - 1
# Round multipliers and Weyl key increments of Philox4x64 (SC'11, Table 2).
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B


def philox4x64_10(counter, key):
    """One Philox4x64 block with 10 rounds: counter (4 x u64), key (2 x u64) -> 4 x u64."""
    c0, c1, c2, c3 = (int(v) & MASK64 for v in counter)
    k0, k1 = (int(v) & MASK64 for v in key)
    for _ in range(10):
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> 64, p0 & MASK64
        hi1, lo1 = p1 >> 64, p1 & MASK64
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        k0 = (k0 + PHILOX_W0) & MASK64
        k1 = (k1 + PHILOX_W1) & MASK64
    return c0, c1, c2, c3


def permutation_draw(seed, signal, m, N):
    """(sigma, a) of iteration m (1-based) of signal ``signal`` for transform size N.

    Block = Philox4x64-10(counter=(signal, m, 0, 0), key=(seed, 0)).
    sigma = 2 * (r0 mod N/2) + 1 (odd, hence invertible mod N = 2^n), a = r1 mod N.
    """
    r = philox4x64_10((signal, m, 0, 0), (seed, 0))
    sigma = 2 * (r[0] % (N // 2)) + 1
    a = r[1] % N
    return sigma, a
