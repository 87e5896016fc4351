"""The vertex order of the GPU forward, modelled on the host: walk P1's
edges in order; edge i emits its start vertex when that vertex is inside P2,
then its entry crossing, then its exit crossing followed by the P2 vertices
after the crossed P2 edge for as long as they are inside P1; with no P1
vertex inside and no crossing, the intersection is P2.  The cycle is then
rotated to start at its smallest code.  No sort and no angle: on polygons in
general position the codes must equal the oracle's, which sorts the
candidates by angle about their centroid."""
import numpy as np
import pytest

from paper_2011_11134_gb300 import workloads as W


def cross(ax, ay, bx, by):
    return ax * by - ay * bx


def walk_codes(p, q, n1, n2, K):
    o = p[0]
    a = p[:n1].astype(np.float64) - o
    b = q[:n2].astype(np.float64) - o
    ea = np.roll(a, -1, axis=0) - a
    eb = np.roll(b, -1, axis=0) - b
    L = max(np.abs(a).max(), np.abs(b).max())
    S = np.array([[cross(*eb[j], *(a[i] - b[j])) for j in range(n2)] for i in range(n1)])
    T = np.array([[cross(*ea[i], *(b[j] - a[i])) for j in range(n2)] for i in range(n1)])
    if min(np.abs(S).min(), np.abs(T).min()) <= 1e-9 * L * L:
        return None
    in1 = (S > 0).all(axis=1)
    in2 = (T > 0).all(axis=0)
    seq = []
    any_cross = False
    for i in range(n1):
        i1 = (i + 1) % n1
        if in1[i]:
            seq.append(i)
        entry = exit_ = None
        for j in range(n2):
            if (T[i, j] > 0) != (T[i, (j + 1) % n2] > 0) and (S[i, j] > 0) != (S[i1, j] > 0):
                any_cross = True
                if S[i, j] < 0:
                    entry = j  # a_i outside P2 edge j, a_i+1 inside: entering
                else:
                    exit_ = j
        if entry is not None:
            seq.append(0x80 | (i << 3) | entry)
        if exit_ is not None:
            seq.append(0x80 | (i << 3) | exit_)
            j = (exit_ + 1) % n2
            while in2[j]:
                seq.append(0x40 | j)
                j = (j + 1) % n2
    if not any_cross and not in1.any():
        seq = [0x40 | j for j in range(n2)] if in2.all() else []
    if len(seq) < 3:
        return [0xFF] * (2 * K)
    r = seq.index(min(seq))
    seq = seq[r:] + seq[:r]
    return seq + [0xFF] * (2 * K - len(seq))


@pytest.mark.parametrize("K", [4, 8])
def test_walk_order_equals_oracle_codes(orc, K):
    if K == 4:
        d = W.loss_pairs_1m(seed=25, n=3000)
        p1, p2 = d["p1"], d["p2"]
        c1 = c2 = np.full(len(p1), 4, np.uint8)
        ref = orc.iou_paired(p1, p2)
    else:
        d = W.convex_pairs_4m(seed=26, n=3000, degenerate_frac=0.0)
        p1, p2, c1, c2 = d["p1"], d["p2"], d["c1"], d["c2"]
        ref = orc.iou_paired(p1, p2, c1, c2)
    checked = 0
    for k in range(len(p1)):
        if ref["degen"][k]:
            continue
        codes = walk_codes(p1[k], p2[k], int(c1[k]), int(c2[k]), K)
        if codes is None:
            continue
        assert codes == ref["xflags"][k].tolist(), (k, codes, ref["xflags"][k].tolist())
        checked += 1
    assert checked > 2000
    assert (ref["nx"] >= 3).sum() > 1000
