"""Pins for the oracle's GIoU / DIoU loss terms (the generalized and
distance-penalised IoU losses over rotated boxes, the IoU-loss case study of
the paper, Sec. IV-A).

The hull area is checked against a closed form for axis-aligned boxes,
containment, and an exact rational gift-wrapping hull (a different algorithm
from the oracle's monotone chain); the centre distance and the diameter
against translated copies whose values are known; the gradients against
central differences of the oracle's own loss term in FP64 and against the
invariances of both losses (translation, rotation, scale).
"""
import math
from fractions import Fraction as F

import numpy as np
import pytest

from paper_2011_11134_gb300 import workloads as W

GIOU, DIOU = 1, 2


def _box(x0, y0, x1, y1):
    return np.array([(x0, y0), (x1, y0), (x1, y1), (x0, y1)], np.float32)


def test_hull_area_axis_aligned_closed_form(orc):
    """Box B2 up and to the right of B1 (x1 < u1, x2 < u2, y1 < v1, y2 < v2):
    the hull is their bounding box less two corner triangles,
    A_h = bbox - (u1 - x1)(v2 - y2) / 2 - (u2 - x2)(v1 - y1) / 2."""
    r = np.random.default_rng(1)
    P, Q, want = [], [], []
    for _ in range(300):
        x1, y1 = r.integers(0, 8, 2)
        x2, y2 = x1 + r.integers(1, 6), y1 + r.integers(1, 6)
        u1, v1 = x1 + r.integers(1, 6), y1 + r.integers(1, 6)
        u2, v2 = max(u1 + 1, x2 + r.integers(1, 4)), max(v1 + 1, y2 + r.integers(1, 4))
        P.append(_box(x1, y1, x2, y2))
        Q.append(_box(u1, v1, u2, v2))
        bbox = (u2 - x1) * (v2 - y1)
        want.append(bbox - 0.5 * (u1 - x1) * (v2 - y2) - 0.5 * (u2 - x2) * (v1 - y1))
    o = orc.loss_variant_paired(np.stack(P), np.stack(Q), GIOU)
    assert np.abs(o["terms"][:, 1] - np.array(want)).max() <= 1e-12 * max(want)


def test_containment_and_identity(orc):
    """Q inside P: the hull is P, so GIoU = IoU = A_2 / A_1; identical boxes:
    both losses are 0 with zero gradient."""
    P = _box(0, 0, 4, 3)
    Q = _box(1, 0.5, 2.5, 2)
    o = orc.loss_variant_paired(P[None], Q[None], GIOU)
    assert o["terms"][0, 1] == pytest.approx(12.0, abs=1e-12)
    assert o["lk"][0] == pytest.approx(1.0 - 2.25 / 12.0, abs=1e-12)
    for v in (GIOU, DIOU):
        o = orc.loss_variant_paired(P[None], P[None], v)
        assert abs(o["lk"][0]) <= 1e-12


def _gift_wrap_area(pts):
    """Exact area of the convex hull of pts (gift wrapping in Fraction)."""
    Pf = sorted({(F(float(x)), F(float(y))) for x, y in pts})
    start = Pf[0]
    hull = [start]
    cur = start
    while True:
        cand = None
        for p in Pf:
            if p == cur:
                continue
            if cand is None:
                cand = p
                continue
            o = (cand[0] - cur[0]) * (p[1] - cur[1]) - (cand[1] - cur[1]) * (p[0] - cur[0])
            far = (p[0] - cur[0]) ** 2 + (p[1] - cur[1]) ** 2 > (cand[0] - cur[0]) ** 2 + (cand[1] - cur[1]) ** 2
            if o < 0 or (o == 0 and far):  # p is right of cur -> cand, or further along the same line
                cand = p
        cur = cand
        if cur == start:
            break
        hull.append(cur)
    return sum(hull[k][0] * hull[(k + 1) % len(hull)][1] - hull[k][1] * hull[(k + 1) % len(hull)][0]
               for k in range(len(hull))) / 2


@pytest.mark.parametrize("K", [4, 8])
def test_hull_area_exact_rational(orc, K):
    """Hull area equals an exact rational gift-wrapping hull of the n1 + n2
    vertices, within double rounding."""
    if K == 4:
        d = W.paired_rect_4096(seed=6, n=200)
        c1 = c2 = None
    else:
        d = W.convex_pairs_4m(seed=6, n=200, degenerate_frac=0.0)
        c1, c2 = d["c1"], d["c2"]
    o = orc.loss_variant_paired(d["p1"], d["p2"], GIOU, c1=c1, c2=c2)
    for k in range(200):
        n1 = K if c1 is None else int(c1[k])
        n2 = K if c2 is None else int(c2[k])
        pts = list(d["p1"][k, :n1]) + list(d["p2"][k, :n2])
        want = float(_gift_wrap_area(pts))
        assert abs(o["terms"][k, 1] - want) <= 1e-12 * max(1.0, want), k


def test_centre_distance_and_diameter_of_translated_copies(orc):
    """Q = P translated by (dx, dy) >= 0, P an axis-aligned w x h box: the
    vertex means are (dx, dy) apart and the diameter runs from P's lower-left
    corner to Q's upper-right corner, c2 = (w + dx)^2 + (h + dy)^2; both hold
    after any rotation of the pair."""
    r = np.random.default_rng(3)
    for _ in range(200):
        w, h = r.uniform(0.5, 4, 2)
        dx, dy = r.uniform(0, 3, 2)
        th = r.uniform(-math.pi, math.pi)
        R = np.array([[math.cos(th), -math.sin(th)], [math.sin(th), math.cos(th)]])
        P = _box(0, 0, w, h).astype(np.float64)
        Q = P + np.array([dx, dy])
        P32, Q32 = (P @ R.T).astype(np.float32), (Q @ R.T).astype(np.float32)
        o = orc.loss_variant_paired(P32[None], Q32[None], DIOU)
        # exact values of the rounded inputs
        m = Q32.astype(np.float64).mean(0) - P32.astype(np.float64).mean(0)
        assert o["terms"][0, 2] == pytest.approx(m @ m, rel=1e-12)
        assert o["terms"][0, 2] == pytest.approx(dx * dx + dy * dy, rel=1e-5, abs=1e-9)
        assert o["terms"][0, 3] == pytest.approx((w + dx) ** 2 + (h + dy) ** 2, rel=1e-5)


def _fd(orc, P, Q, v, K, h_rel=1e-6):
    lk, g1, g2 = orc.loss_variant_pair_f64(P, Q, v, 1.0, K)
    L = max(np.abs(P - P[0]).max(), np.abs(Q - P[0]).max())
    h = h_rel * L
    num = [np.zeros_like(P), np.zeros_like(Q)]
    for which in (0, 1):
        for vv in range((P, Q)[which].shape[0]):
            for c in range(2):
                vals = []
                for sgn in (1, -1):
                    A, B = P.copy(), Q.copy()
                    (A if which == 0 else B)[vv, c] += sgn * h
                    vals.append(orc.loss_variant_pair_f64(A, B, v, 1.0, K)[0])
                num[which][vv, c] = (vals[0] - vals[1]) / (2 * h)
    return (g1, g2), num


@pytest.mark.parametrize("v", [GIOU, DIOU])
@pytest.mark.parametrize("K", [4, 8])
def test_finite_differences(orc, v, K):
    """Gradient of the loss term = central differences of the oracle's loss
    term in FP64, on pairs the oracle does not flag near-degenerate (and, for
    DIoU, whose diameter is not a near-tie)."""
    if K == 4:
        d = W.loss_pairs_1m(seed=9, n=150)
        c1 = c2 = None
    else:
        d = W.convex_pairs_4m(seed=9, n=150, degenerate_frac=0.0)
        c1, c2 = d["c1"], d["c2"]
    f = orc.iou_paired(d["p1"], d["p2"], c1, c2)
    checked = 0
    for k in range(150):
        if f["degen"][k]:
            continue
        n1 = K if c1 is None else int(c1[k])
        n2 = K if c2 is None else int(c2[k])
        P = d["p1"][k, :n1].astype(np.float64)
        Q = d["p2"][k, :n2].astype(np.float64)
        if v == DIOU:
            # the diameter is a maximum over vertex pairs: where the two largest
            # distances nearly tie (a rectangle's two diagonals) it has no
            # derivative, so such pairs are skipped
            pts = np.concatenate([P, Q])
            dd = np.sort(((pts[:, None, :] - pts[None, :, :]) ** 2).sum(-1)[np.triu_indices(len(pts), 1)])
            if dd[-1] - dd[-2] < 1e-4 * dd[-1]:
                continue
        (g1, g2), (n1v, n2v) = _fd(orc, P, Q, v, K)
        G = np.concatenate([g1, g2])
        N = np.concatenate([n1v, n2v])
        assert np.abs(G - N).max() <= 1e-5 * max(np.abs(N).max(), 1e-3), k
        checked += 1
    assert checked >= 50


@pytest.mark.parametrize("v", [GIOU, DIOU])
def test_gradient_invariants(orc, v):
    """Both losses are invariant to translating, rotating and scaling the pair
    together, so over all vertices sum g = 0, sum cross(p, g) = 0 and
    sum p . g = 0."""
    d = W.convex_pairs_4m(seed=12, n=300, degenerate_frac=0.0)
    o = orc.loss_variant_paired(d["p1"], d["p2"], v, c1=d["c1"], c2=d["c2"])
    for k in range(300):
        n1, n2 = int(d["c1"][k]), int(d["c2"][k])
        pts = np.concatenate([d["p1"][k, :n1], d["p2"][k, :n2]]).astype(np.float64)
        g = np.concatenate([o["g1"][k, :n1], o["g2"][k, :n2]])
        scale = np.abs(g).max() * np.abs(pts).max() + 1e-30
        assert np.abs(g.sum(0)).max() <= 1e-10 * np.abs(g).max() + 1e-300
        assert abs((pts[:, 0] * g[:, 1] - pts[:, 1] * g[:, 0]).sum()) <= 1e-9 * scale
        assert abs((pts * g).sum()) <= 1e-9 * scale


def test_weights_scale_the_terms(orc):
    d = W.paired_rect_4096(seed=1, n=50)
    w = np.linspace(0.5, 2.0, 50)
    for v in (GIOU, DIOU):
        a = orc.loss_variant_paired(d["p1"], d["p2"], v)
        b = orc.loss_variant_paired(d["p1"], d["p2"], v, weight=w)
        assert np.allclose(b["lk"], w * a["lk"], rtol=1e-14, atol=0)
        assert np.allclose(b["g1"], w[:, None, None] * a["g1"], rtol=1e-13, atol=1e-300)
