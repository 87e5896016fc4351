"""Host model of the backward's piece-count check for quadrilaterals.

The K = 4 backward tests the crossings recorded for a pair against the
inside vertices with bit-parallel arithmetic on 4-bit fields (one field per
edge, rows of the 4 x 4 crossing mask for P1's edges, its transpose for
P2's).  This checks, for every inside mask and every crossing mask, that the
bit-parallel form accepts exactly what the per-edge rule accepts: an edge
whose ends are one inside and one outside carries one crossing, an edge with
both ends inside carries none, an edge with both ends outside carries none or
two (a chord of the other polygon)."""
import numpy as np


def _per_edge(in1, in2, X):
    ok = np.ones(X.shape, bool)
    for i in range(4):
        ra = sum((X >> (4 * i + j)) & 1 for j in range(4))
        a0, a1 = (in1 >> i) & 1, (in1 >> ((i + 1) % 4)) & 1
        ok &= np.where(a0 ^ a1, ra == 1, np.where(a0 == 1, ra == 0, (ra == 0) | (ra == 2)))
        rb = sum((X >> (4 * j + i)) & 1 for j in range(4))
        b0, b1 = (in2 >> i) & 1, (in2 >> ((i + 1) % 4)) & 1
        ok &= np.where(b0 ^ b1, rb == 1, np.where(b0 == 1, rb == 0, (rb == 0) | (rb == 2)))
    return ok


def _bit_parallel(in1, in2, X):
    x = X.astype(np.uint32)
    t = (x ^ (x >> 3)) & 0x0A0A
    xt = x ^ t ^ (t << 3)
    t = (xt ^ (xt >> 6)) & 0x00CC
    xt = xt ^ t ^ (t << 6)

    def nib_pop(v):
        v = (v & 0x5555) + ((v >> 1) & 0x5555)
        return (v & 0x3333) + ((v >> 2) & 0x3333)

    def spread(m):
        return (m | (m << 3) | (m << 6) | (m << 9)) & 0x1111

    in1n = ((in1 >> 1) | (in1 << 3)) & 15
    in2n = ((in2 >> 1) | (in2 << 3)) & 15
    mask32 = np.uint32(0xFFFFFFFF)
    da = (nib_pop(x) ^ spread(in1 ^ in1n)) & (mask32 ^ (spread(~(in1 | in1n) & 15) << 1))
    db = (nib_pop(xt) ^ spread(in2 ^ in2n)) & (mask32 ^ (spread(~(in2 | in2n) & 15) << 1))
    return (da | db) == 0


def test_transpose_moves_every_bit():
    for i in range(4):
        for j in range(4):
            x = np.array([1 << (4 * i + j)], np.uint32)
            t = (x ^ (x >> 3)) & 0x0A0A
            xt = x ^ t ^ (t << 3)
            t = (xt ^ (xt >> 6)) & 0x00CC
            xt = xt ^ t ^ (t << 6)
            assert int(xt[0]) == 1 << (4 * j + i)


def test_bit_parallel_rule_equals_per_edge_rule():
    X = np.arange(1 << 16, dtype=np.uint32)
    accepted = 0
    for in1 in range(16):
        for in2 in range(16):
            a = np.uint32(in1)
            b = np.uint32(in2)
            want = _per_edge(a, b, X)
            got = _bit_parallel(a, b, X)
            assert np.array_equal(want, got), (in1, in2, np.flatnonzero(want != got)[:5])
            accepted += int(want.sum())
    assert accepted > 0
