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



def model_grads(p, q, n1, n2, g=1.0):
    """dL/dP1, dL/dP2 for L = g IoU by the backward's shape derivative (FP64):
    each clipped edge piece [t0, t1] moves with its edge's endpoints, so edge v
    adds (g_Ai I0 + g_A/2) n_v to its start vertex and (g_Ai I1 + g_A/2) n_v to
    its end vertex, with n_v = (ey, -ex), I0 = ((1-t0)^2 - (1-t1)^2) / 2 and
    I1 = (t1^2 - t0^2) / 2 (the integrals of 1 - t and t over the piece).
    None when not in general position or the polygons do not overlap."""
    o = p[0]
    a = p[:n1] - o
    b = q[:n2] - o
    ea = np.roll(a, -1, axis=0) - a
    eb = np.roll(b, -1, axis=0) - b
    L = max(np.abs(a).max(), np.abs(b).max())
    S = np.array([[cross(*eb[j], *(a[i] - b[j])) for j in range(n2)] for i in range(n1)])
    T = np.array([[cross(*ea[i], *(b[j] - a[i])) for j in range(n2)] for i in range(n1)])
    if min(np.abs(S).min(), np.abs(T).min()) <= 1e-9 * L * L:
        return None
    in1 = (S > 0).all(axis=1)
    in2 = (T > 0).all(axis=0)
    t0, t1 = np.full(n1, np.inf), np.full(n1, -np.inf)
    u0, u1 = np.full(n2, np.inf), np.full(n2, -np.inf)
    hasA, hasB = in1.copy(), in2.copy()
    for i in range(n1):
        for j in range(n2):
            if (S[i, j] > 0) != (S[(i + 1) % n1, j] > 0) and (T[i, j] > 0) != (T[i, (j + 1) % n2] > 0):
                D = cross(*ea[i], *eb[j])
                t, u = S[i, j] / D, -T[i, j] / D
                t0[i], t1[i] = min(t0[i], t), max(t1[i], t)
                u0[j], u1[j] = min(u0[j], u), max(u1[j], u)
                hasA[i] = hasB[j] = True
    if not (hasA.any() or hasB.any()):
        return None
    t0 = np.where(in1, 0.0, t0)
    t1 = np.where(np.roll(in1, -1), 1.0, t1)
    u0 = np.where(in2, 0.0, u0)
    u1 = np.where(np.roll(in2, -1), 1.0, u1)
    # edges with no piece: any finite placeholder (their terms are masked out)
    t0, t1 = np.where(hasA, t0, 0.0), np.where(hasA, t1, 0.0)
    u0, u1 = np.where(hasB, u0, 0.0), np.where(hasB, u1, 0.0)
    c1 = np.array([cross(*a[v], *ea[v]) for v in range(n1)])
    c2 = np.array([cross(*b[v], *eb[v]) for v in range(n2)])
    two = np.where(hasA, (t1 - t0) * c1, 0.0).sum() + np.where(hasB, (u1 - u0) * c2, 0.0).sum()
    ai, a1, a2 = 0.5 * two, 0.5 * c1.sum(), 0.5 * c2.sum()
    U = a1 + a2 - ai
    if ai <= 0 or U <= 0:
        return None
    gai, gA = g * (a1 + a2) / U**2, -g * ai / U**2  # dIoU/dA_i, dIoU/dA_1 = dIoU/dA_2

    def vertex_grads(e, s0, s1, has, n):
        I0 = np.where(has, 0.5 * ((1 - s0) ** 2 - (1 - s1) ** 2), 0.0)
        I1 = np.where(has, 0.5 * (s1**2 - s0**2), 0.0)
        nv = np.stack([e[:, 1], -e[:, 0]], 1)
        start = (gai * I0 + 0.5 * gA)[:, None] * nv
        end = (gai * I1 + 0.5 * gA)[:, None] * nv
        return start + np.roll(end, 1, axis=0)

    return vertex_grads(ea, t0, t1, hasA, n1), vertex_grads(eb, u0, u1, hasB, n2)


@pytest.mark.parametrize("K", [4, 8])
def test_shape_derivative_equals_oracle_adjoint(orc, K):
    """The backward's shape derivative (no crossing points, no reverse pass
    through the clip) gives the gradient of the oracle's shoelace adjoint."""
    if K == 4:
        d = W.loss_pairs_1m(seed=23, n=1500)
        p1, p2 = d["p1"], d["p2"]
        c1 = c2 = np.full(len(p1), 4, np.uint8)
        ref = orc.iou_paired(p1, p2)
        o1, o2 = orc.iou_backward_paired(p1, p2, np.ones(len(p1)), ref["nx"], ref["xflags"])
    else:
        d = W.convex_pairs_4m(seed=24, n=1500, degenerate_frac=0.0)
        p1, p2, c1, c2 = d["p1"], d["p2"], d["c1"], d["c2"]
        ref = orc.iou_paired(p1, p2, c1, c2)
        o1, o2 = orc.iou_backward_paired(p1, p2, np.ones(len(p1)), ref["nx"], ref["xflags"], c1, c2)
    checked = 0
    for k in range(len(p1)):
        if ref["degen"][k] or ref["nx"][k] < 3:
            continue
        m = model_grads(p1[k].astype(np.float64), p2[k].astype(np.float64), int(c1[k]), int(c2[k]))
        if m is None:
            continue
        g1, g2 = m
        n1, n2 = int(c1[k]), int(c2[k])
        scale = max(np.abs(o1[k]).max(), np.abs(o2[k]).max(), 1e-6)
        err = max(np.abs(g1 - o1[k, :n1]).max(), np.abs(g2 - o2[k, :n2]).max()) / scale
        assert err <= 1e-8, (k, err)
        checked += 1
    assert checked > 800
