"""The area formula of the GPU forward, modelled in FP64 on the host, equals
the shoelace area of the intersection polygon that the oracle builds.

The forward never forms a crossing point.  Twice the intersection area is
taken as a sum over edge pieces, in P1's local frame (origin at P1's vertex
0), with S(i, j) = orient(b_j, b_j+1, a_i), T(i, j) = orient(a_i, a_i+1, b_j)
and D(i, j) = cross(ea_i, eb_j):
  * each P1 vertex a_i+1 inside P2 adds cross(a_i, ea_i), and each P2 vertex
    b_j+1 inside P1 adds cross(b_j, eb_j);
  * each proper crossing of P1 edge i with P2 edge j adds
    (cross(a_i, b_j) D + S T) / |D|.
Both sides of the identity are evaluated here in FP64 from the same float
inputs, on polygons in general position (no orientation within 1e-9 L^2 of
zero), so the two must agree to rounding."""
import numpy as np
import pytest

from paper_2011_11134_gb300 import workloads as W


def cross(ax, ay, bx, by):
    return ax * by - ay * bx


def model_two_area(p, q, n1, n2):
    """2 A_i by the forward's formula (FP64), or None if the pair is not in
    general position."""
    o = p[0]
    a = p[:n1] - o
    b = q[:n2] - o
    ea = np.roll(a, -1, axis=0) - a
    eb = np.roll(b, -1, axis=0) - b
    L = max(np.abs(a).max(), np.abs(b).max())
    S = np.zeros((n1, n2))
    T = np.zeros((n1, n2))
    for i in range(n1):
        for j in range(n2):
            S[i, j] = cross(eb[j, 0], eb[j, 1], a[i, 0] - b[j, 0], a[i, 1] - b[j, 1])
            T[i, j] = cross(ea[i, 0], ea[i, 1], b[j, 0] - a[i, 0], b[j, 1] - a[i, 1])
    if min(np.abs(S).min(), np.abs(T).min()) <= 1e-9 * L * L:
        return None
    in1 = (S > 0).all(axis=1)  # P1 vertex i inside P2
    in2 = (T > 0).all(axis=0)  # P2 vertex j inside P1
    two = 0.0
    for v in range(n1):
        if in1[(v + 1) % n1]:
            two += cross(a[v, 0], a[v, 1], ea[v, 0], ea[v, 1])
    for v in range(n2):
        if in2[(v + 1) % n2]:
            two += cross(b[v, 0], b[v, 1], eb[v, 0], eb[v, 1])
    for i in range(n1):
        i1 = (i + 1) % n1
        for j in range(n2):
            j1 = (j + 1) % n2
            # strict sign change along both edges: a proper crossing
            if (S[i, j] > 0) != (S[i1, j] > 0) and (T[i, j] > 0) != (T[i, j1] > 0):
                D = cross(ea[i, 0], ea[i, 1], eb[j, 0], eb[j, 1])
                c = cross(a[i, 0], a[i, 1], b[j, 0], b[j, 1])
                two += (c * D + S[i, j] * T[i, j]) / abs(D)
    return two


@pytest.mark.parametrize("K", [4, 8])
def test_crossing_term_area_equals_shoelace(orc, K):
    if K == 4:
        d = W.loss_pairs_1m(seed=21, n=3000)
        p1, p2 = d["p1"], d["p2"]
        c1 = c2 = np.full(len(p1), 4, np.uint8)
    else:
        d = W.convex_pairs_4m(seed=22, n=3000, degenerate_frac=0.0)
        p1, p2, c1, c2 = d["p1"], d["p2"], d["c1"], d["c2"]
    ref = orc.iou_paired(p1, p2, None if K == 4 else c1, None if K == 4 else c2)
    checked = 0
    for k in range(len(p1)):
        two = model_two_area(p1[k].astype(np.float64), p2[k].astype(np.float64), int(c1[k]), int(c2[k]))
        if two is None:
            continue
        L = max(np.abs(p1[k] - p1[k, 0]).max(), np.abs(p2[k] - p1[k, 0]).max())
        ai = ref["areas"][k, 0]
        got = 0.5 * two if ref["nx"][k] >= 3 else 0.0
        assert abs(got - ai) <= 1e-9 * L * L, (k, got, ai)
        checked += 1
    assert checked > 2500
    assert (ref["nx"] >= 3).sum() > 1000  # most pairs overlap

