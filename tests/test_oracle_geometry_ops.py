"""Pins for the oracle's exported geometry operations: `intersect` (the
intersection polygon's vertices), `area`, and the line operations (paper
Sec. II-B listing and Sec. III "Lines").  Each is checked against something
other than itself: exact rational clipping, closed forms, and central
differences of the forward."""
import numpy as np
import pytest

from paper_2011_11134_gb300 import workloads as W

from . import exact_clip


@pytest.mark.parametrize("K", [4, 8])
def test_intersect_vertices_match_exact_clip(orc, K):
    """Every vertex of the oracle's intersection polygon is, within double
    rounding, a vertex of the exact rational clip, in counter-clockwise order,
    and the vertex count matches."""
    if K == 4:
        d = W.paired_rect_4096(seed=11, n=200)
        p1, p2, c1, c2 = d["p1"], d["p2"], None, None
    else:
        d = W.convex_pairs_4m(seed=11, n=200, degenerate_frac=0.0)
        p1, p2, c1, c2 = d["p1"], d["p2"], d["c1"], d["c2"]
    o = orc.intersect_paired(p1, p2, c1, c2)
    ref = orc.iou_paired(p1, p2, c1, c2)
    assert (o["nx"] == ref["nx"]).all() and (o["xflags"] == ref["xflags"]).all()
    checked = 0
    for k in range(p1.shape[0]):
        n1 = K if c1 is None else int(c1[k])
        n2 = K if c2 is None else int(c2[k])
        inter = exact_clip.clip([tuple(v) for v in p1[k, :n1]], [tuple(v) for v in p2[k, :n2]])
        nx = int(o["nx"][k])
        assert (o["verts"][k, nx:] == 0).all()
        if ref["degen"][k] or nx == 0:
            continue
        # the exact clip may repeat a point: distinct exact points
        ex = np.array([[float(x), float(y)] for x, y in sorted(set(inter))])
        got = o["verts"][k, :nx]
        assert len(ex) == nx, k
        # crossing points are a + t (b - a) in double; away from nearly
        # parallel edges (flagged near-degenerate, skipped above) their error
        # is well under 1e-10 of the coordinates
        L = max(1.0, np.abs(got).max())
        for v in got:
            assert np.abs(ex - v).max(1).min() <= 1e-10 * L, k
        # counter-clockwise: every consecutive triple turns left
        nxt, nn = np.roll(got, -1, 0), np.roll(got, -2, 0)
        turn = (nxt[:, 0] - got[:, 0]) * (nn[:, 1] - got[:, 1]) - (nxt[:, 1] - got[:, 1]) * (nn[:, 0] - got[:, 0])
        assert (turn > 0).all(), k
        checked += 1
    assert checked > 120


def test_intersect_axis_aligned_closed_form(orc):
    """Two axis-aligned rectangles intersect in the rectangle of the inner
    bounds: its four corners, counter-clockwise."""
    r = np.random.default_rng(12)
    n = 300
    lo1, lo2 = r.uniform(0, 4, (n, 2)), r.uniform(0, 4, (n, 2))
    hi1, hi2 = lo1 + r.uniform(1, 4, (n, 2)), lo2 + r.uniform(1, 4, (n, 2))

    def rect(lo, hi):
        return np.stack([lo, np.stack([hi[:, 0], lo[:, 1]], 1), hi, np.stack([lo[:, 0], hi[:, 1]], 1)], 1)

    p1 = rect(lo1, hi1).astype(np.float32)
    p2 = rect(lo2, hi2).astype(np.float32)
    o = orc.intersect_paired(p1, p2)
    L = np.maximum(p1.astype(np.float64).min(1), p2.astype(np.float64).min(1))
    H = np.minimum(p1.astype(np.float64).max(1), p2.astype(np.float64).max(1))
    for k in range(n):
        if (H[k] <= L[k]).any():
            assert o["nx"][k] == 0
            continue
        want = np.array([[L[k, 0], L[k, 1]], [H[k, 0], L[k, 1]], [H[k, 0], H[k, 1]], [L[k, 0], H[k, 1]]])
        got = o["verts"][k, :o["nx"][k]]
        assert len(got) == 4, k
        # crossing points carry the rounding of a + t (b - a)
        for v in got:
            assert np.abs(want - v).max(1).min() <= 1e-14 * 10, k
        # counter-clockwise
        assert 0.5 * np.sum(got[:, 0] * np.roll(got[:, 1], -1) - np.roll(got[:, 0], -1) * got[:, 1]) > 0


def test_area_closed_forms(orc):
    d = W.paired_rect_4096(seed=13, n=500)
    # rotated rectangle from its own corners: |e0| |e1|
    p = d["p1"].astype(np.float64)
    w = np.hypot(*(p[:, 1] - p[:, 0]).T)
    h = np.hypot(*(p[:, 2] - p[:, 1]).T)
    assert np.allclose(orc.area(d["p1"]), w * h, rtol=1e-6, atol=0)
    # triangles with counts: half the cross product of two edges
    c = W.convex_pairs_4m(seed=13, n=500, degenerate_frac=0.0)
    tri = c["c1"] == 3
    assert tri.any()
    q = c["p1"][tri].astype(np.float64)
    want = 0.5 * ((q[:, 1, 0] - q[:, 0, 0]) * (q[:, 2, 1] - q[:, 0, 1]) - (q[:, 1, 1] - q[:, 0, 1]) * (q[:, 2, 0] - q[:, 0, 0]))
    assert np.allclose(orc.area(c["p1"], c["c1"])[tri], want, rtol=1e-12, atol=1e-12)
    bad = c["c1"].copy()
    bad[0] = 2
    assert orc.area(c["p1"], bad)[0] == 0.0


def test_lines_closed_forms(orc):
    r = np.random.default_rng(14)
    p, q = r.uniform(-5, 5, (400, 2)), r.uniform(-5, 5, (400, 2))
    ln = orc.line_from_points(p, q)
    for pt in (p, q):
        res = ln[:, 0] * pt[:, 0] + ln[:, 1] * pt[:, 1] + ln[:, 2]
        assert np.abs(res).max() <= 1e-12 * 100
    # the diagonals of the square (0,0)-(2,2) meet at (1, 1); the axes at 0
    d1 = orc.line_from_points(np.array([[0.0, 0.0]]), np.array([[2.0, 2.0]]))
    d2 = orc.line_from_points(np.array([[0.0, 2.0]]), np.array([[2.0, 0.0]]))
    assert np.allclose(orc.line_intersect(d1, d2), [[1.0, 1.0]], atol=1e-15)
    xa = np.array([[0.0, 1.0, 0.0]])  # y = 0
    ya = np.array([[1.0, 0.0, 0.0]])  # x = 0
    assert np.allclose(orc.line_intersect(xa, ya), [[0.0, 0.0]], atol=0)
    # the intersection of two random lines lies on both
    r2, s2 = r.uniform(-5, 5, (400, 2)), r.uniform(-5, 5, (400, 2))
    m = orc.line_from_points(r2, s2)
    x = orc.line_intersect(ln, m)
    ok = np.abs(ln[:, 0] * m[:, 1] - m[:, 0] * ln[:, 1]) > 1e-2
    for l_ in (ln, m):
        res = l_[:, 0] * x[:, 0] + l_[:, 1] * x[:, 1] + l_[:, 2]
        assert np.abs(res[ok]).max() <= 1e-9 * np.abs(x[ok]).max() * 100
    # parallel lines: non-finite
    assert not np.isfinite(orc.line_intersect(xa, np.array([[0.0, 2.0, 1.0]]))).all()


def test_lines_gradients_central_differences(orc):
    r = np.random.default_rng(15)
    n = 50
    p, q = r.uniform(-5, 5, (n, 2)), r.uniform(-5, 5, (n, 2))
    g = r.normal(size=(n, 3))
    gp, gq = orc.line_from_points_backward(p, q, g)
    h = 1e-6
    for arr, ga in ((p, gp), (q, gq)):
        for c in range(2):
            e = np.zeros_like(arr)
            e[:, c] = h
            up = orc.line_from_points(p + e if arr is p else p, q + e if arr is q else q)
            dn = orc.line_from_points(p - e if arr is p else p, q - e if arr is q else q)
            fd = ((up - dn) / (2 * h) * g).sum(1)
            assert np.allclose(ga[:, c], fd, rtol=1e-6, atol=1e-8)
    l1 = orc.line_from_points(p, q)
    l2 = orc.line_from_points(r.uniform(-5, 5, (n, 2)), r.uniform(-5, 5, (n, 2)))
    keep = np.abs(l1[:, 0] * l2[:, 1] - l2[:, 0] * l1[:, 1]) > 1.0
    l1, l2 = l1[keep], l2[keep]
    gx = r.normal(size=(l1.shape[0], 2))
    g1, g2 = orc.line_intersect_backward(l1, l2, gx)
    for arr, ga in ((l1, g1), (l2, g2)):
        for c in range(3):
            e = np.zeros_like(arr)
            e[:, c] = h
            up = orc.line_intersect(l1 + e if arr is l1 else l1, l2 + e if arr is l2 else l2)
            dn = orc.line_intersect(l1 - e if arr is l1 else l1, l2 - e if arr is l2 else l2)
            fd = ((up - dn) / (2 * h) * gx).sum(1)
            assert np.allclose(ga[:, c], fd, rtol=1e-5, atol=1e-7)
