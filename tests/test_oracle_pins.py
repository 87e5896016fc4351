"""Pins for the FP64 oracle against results it does not compute itself.

Each test checks the oracle against something the mathematics fixes: hand
worked cases, closed forms, exact rational clipping by a different
algorithm, point sampling, finite differences, invariances.  Together they
are chosen so that a dropped term, a wrong sign or index, or a transposed
operand anywhere in the oracle fails at least one of them (see
test_oracle_mutations.py, which plants such mistakes and checks that they
are caught).
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2011_11134_gb300 import workloads as W

from . import exact_clip

HERE = os.path.dirname(os.path.abspath(__file__))


def _pad(poly, K):
    poly = np.asarray(poly, np.float32)
    out = np.repeat(poly[:1], K, axis=0)
    out[: len(poly)] = poly
    return out


def _run_pairs(orc, pairs, K):
    p1 = np.stack([_pad(a, K) for a, _ in pairs])
    p2 = np.stack([_pad(b, K) for _, b in pairs])
    c1 = np.array([len(a) for a, _ in pairs], np.uint8)
    c2 = np.array([len(b) for _, b in pairs], np.uint8)
    return orc.iou_paired(p1, p2, c1, c2), p1, p2, c1, c2


# ------------------------------------------------------------ worked cases


def test_handworked_golden(orc):
    """Hand-derived IoU, areas, nx and codes (tests/golden/handworked.json)."""
    cases = json.load(open(os.path.join(HERE, "golden", "handworked.json")))["cases"]
    K = 4
    out, *_ = _run_pairs(orc, [(c["p1"], c["p2"]) for c in cases], K)
    for k, c in enumerate(cases):
        assert out["iou"][k] == pytest.approx(c["iou"], abs=1e-15), c["name"]
        assert out["areas"][k, 0] == pytest.approx(c["ai"], abs=1e-15)
        assert out["areas"][k, 1] == pytest.approx(c["a1"], abs=1e-15)
        assert out["areas"][k, 2] == pytest.approx(c["a2"], abs=1e-15)
        assert out["nx"][k] == c["nx"], c["name"]
        want = c["codes"] + [0xFF] * (2 * K - len(c["codes"]))
        assert list(out["xflags"][k]) == want, c["name"]


# ------------------------------------------------------------ special cases


def test_identity(orc):
    """IoU(a, a) = 1, nx = K, codes = P1 vertices in order (P1 precedence)."""
    d = W.paired_rect_4096(seed=3, n=500)
    o = orc.iou_paired(d["p1"], d["p1"])
    assert np.abs(o["iou"] - 1).max() <= 1e-12
    assert (o["nx"] == 4).all()
    assert (o["xflags"][:, :4] == np.arange(4)).all() and (o["xflags"][:, 4:] == 0xFF).all()
    assert o["degen"].all()  # identical edges are collinear: always flagged


def test_disjoint(orc):
    """Pairs separated by an axis give IoU 0, nx 0 and all-0xFF flags."""
    d = W.paired_rect_4096(seed=4, n=500)
    p2 = d["p2"].copy()
    shift = (d["p1"][..., 0].max(1) - d["p2"][..., 0].min(1)) + 0.5
    p2[..., 0] += shift[:, None]
    o = orc.iou_paired(d["p1"], p2)
    assert (o["iou"] == 0).all() and (o["nx"] == 0).all() and (o["xflags"] == 0xFF).all()


def test_axis_aligned_closed_form(orc):
    """Axis-aligned rectangles: A_i = max(0, min x2 - max x1) * max(0, min y2 - max y1)."""
    r = W.rng_for(11)
    n = 3000
    lo1 = r.uniform(0, 4, (n, 2))
    hi1 = lo1 + r.uniform(0.2, 3, (n, 2))
    lo2 = lo1 + r.uniform(-2, 2, (n, 2))
    hi2 = lo2 + r.uniform(0.2, 3, (n, 2))

    def rect(lo, hi):
        return np.stack([np.stack([lo[:, 0], lo[:, 1]], -1), np.stack([hi[:, 0], lo[:, 1]], -1),
                         np.stack([hi[:, 0], hi[:, 1]], -1), np.stack([lo[:, 0], hi[:, 1]], -1)], 1).astype(
                             np.float32)

    p1, p2 = rect(lo1, hi1), rect(lo2, hi2)
    o = orc.iou_paired(p1, p2)
    P1, P2 = p1.astype(np.float64), p2.astype(np.float64)
    ix = np.maximum(0, np.minimum(P1[:, 2, 0], P2[:, 2, 0]) - np.maximum(P1[:, 0, 0], P2[:, 0, 0]))
    iy = np.maximum(0, np.minimum(P1[:, 2, 1], P2[:, 2, 1]) - np.maximum(P1[:, 0, 1], P2[:, 0, 1]))
    ai = ix * iy
    a1 = (P1[:, 2, 0] - P1[:, 0, 0]) * (P1[:, 2, 1] - P1[:, 0, 1])
    a2 = (P2[:, 2, 0] - P2[:, 0, 0]) * (P2[:, 2, 1] - P2[:, 0, 1])
    want = ai / (a1 + a2 - ai)
    ok = o["degen"] == 0
    assert ok.sum() > 2000
    np.testing.assert_allclose(o["iou"][ok], want[ok], rtol=0, atol=1e-12)
    np.testing.assert_allclose(o["areas"][ok, 0], ai[ok], rtol=1e-12, atol=1e-12)


def test_rotated_rect_area(orc):
    """A rotated rectangle built from (w, h, theta) has area w*h (shoelace A_1)."""
    r = W.rng_for(12)
    n = 2000
    w, h = r.uniform(0.5, 4, n), r.uniform(0.5, 4, n)
    th = r.uniform(-np.pi, np.pi, n)
    c = r.uniform(0, 10, (n, 2))
    p = W.boxes_to_polygons(c[:, 0], c[:, 1], w, h, th)
    o = orc.iou_paired(p, p)
    # float32 corner rounding perturbs the area by O(ulp(10) * (w + h))
    np.testing.assert_allclose(o["areas"][:, 1], w * h, rtol=2e-6)
    # the exact area of the stored float32 corners, by exact rational shoelace
    for k in range(50):
        ex = exact_clip.area([(x, y) for x, y in p[k]])
        assert abs(float(ex) - o["areas"][k, 1]) <= 1e-12 * max(1.0, float(ex))


def test_nested(orc):
    """P2 inside P1: IoU = A_2 / A_1 and the flags are P2's vertices in order."""
    r = W.rng_for(13)
    n = 1000
    c = r.uniform(0, 10, (n, 2))
    th = r.uniform(-np.pi, np.pi, n)
    w, h = r.uniform(2, 4, n), r.uniform(2, 4, n)
    big = W.boxes_to_polygons(c[:, 0], c[:, 1], w, h, th)
    small = W.boxes_to_polygons(c[:, 0], c[:, 1], 0.5 * w, 0.4 * h, th + r.uniform(-0.3, 0.3, n))
    o = orc.iou_paired(big, small)
    a_big, a_small = o["areas"][:, 1], o["areas"][:, 2]
    np.testing.assert_allclose(o["iou"], a_small / a_big, rtol=1e-12)
    assert (o["nx"] == 4).all()
    assert (o["xflags"][:, :4] == 0x40 + np.arange(4)).all()


# ---------------------------------------------------- symmetry / invariance


def _swap_codes(codes):
    out = []
    for c in codes:
        if c == 0xFF:
            continue
        kind = c >> 6
        if kind == 0:
            out.append(0x40 | c)
        elif kind == 1:
            out.append(c & 0x3F)
        else:
            i, j = (c >> 3) & 7, c & 7
            out.append(0x80 | (j << 3) | i)
    return sorted(out)


def test_symmetry(orc):
    """IoU(a, b) = IoU(b, a); the code set maps by swapping the P1/P2 roles."""
    d = W.paired_rect_4096(seed=5, n=2000)
    o = orc.iou_paired(d["p1"], d["p2"])
    s = orc.iou_paired(d["p2"], d["p1"])
    np.testing.assert_allclose(o["iou"], s["iou"], rtol=0, atol=1e-12)
    gen = (o["degen"] == 0) & (s["degen"] == 0)
    assert gen.sum() > 1900
    for k in np.nonzero(gen)[0][:500]:
        assert _swap_codes(o["xflags"][k]) == sorted(int(c) for c in s["xflags"][k] if c != 0xFF)


def test_rotation_translation_invariance(orc):
    """Jointly rotating both polygons by 90 degrees (exact in float32) and
    translating them by powers of two (exact in double for float32 inputs)
    changes neither IoU nor the codes."""
    d = W.paired_rect_4096(seed=6, n=1000)
    o = orc.iou_paired(d["p1"], d["p2"])

    def rot90(p):
        return np.stack([-p[..., 1], p[..., 0]], -1)

    t = orc.iou_paired(rot90(d["p1"]), rot90(d["p2"]))
    np.testing.assert_allclose(t["iou"], o["iou"], rtol=0, atol=1e-12)
    gen = (o["degen"] == 0) & (t["degen"] == 0)
    assert gen.sum() > 950
    assert (t["xflags"][gen] == o["xflags"][gen]).all()
    assert (t["nx"][gen] == o["nx"][gen]).all()
    for k in range(300):
        P, Q = d["p1"][k].astype(np.float64), d["p2"][k].astype(np.float64)
        for shift in (8.0, -16.0, 1024.0):
            r = orc.iou_pair_f64(P + shift, Q + shift, 4)
            # absolute-coordinate arithmetic: rounding grows with |coordinate|^2
            assert abs(r[0] - o["iou"][k]) <= 1e-12 + 1e-14 * shift * shift
            if not o["degen"][k] and not r[6]:
                assert r[4] == o["nx"][k] and list(r[5]) == list(o["xflags"][k])


# ------------------------------------------------------ independent methods


@pytest.mark.parametrize("K", [4, 8])
def test_exact_rational_clip(orc, K):
    """The oracle's A_i and code sequence equal those of an exact rational
    Sutherland-Hodgman clip (a different algorithm, no rounding)."""
    if K == 4:
        d = W.paired_rect_4096(seed=7, n=300)
        p1, p2, c1, c2 = d["p1"], d["p2"], None, None
    else:
        d = W.convex_pairs_4m(seed=7, n=300, degenerate_frac=0.0)
        p1, p2, c1, c2 = d["p1"], d["p2"], d["c1"], d["c2"]
    o = orc.iou_paired(p1, p2, c1, c2)
    checked = 0
    for k in range(p1.shape[0]):
        n1 = K if c1 is None else int(c1[k])
        n2 = K if c2 is None else int(c2[k])
        P = [tuple(v) for v in p1[k, :n1]]
        Q = [tuple(v) for v in p2[k, :n2]]
        inter = exact_clip.clip(P, Q)
        ai = float(exact_clip.area(inter)) if len(inter) >= 3 else 0.0
        assert abs(o["areas"][k, 0] - ai) <= 1e-12 * max(1.0, abs(ai)), k
        if o["degen"][k]:
            continue
        seq = exact_clip.codes(P, Q, inter)
        assert seq is not None
        got = [int(c) for c in o["xflags"][k] if c != 0xFF]
        assert got == seq, (k, got, seq)
        assert o["nx"][k] == len(seq)
        checked += 1
    assert checked > 250


def test_point_sampling(orc):
    """Monte-Carlo estimate of the intersection area agrees within 4 sigma."""
    d = W.convex_pairs_4m(seed=8, n=40, degenerate_frac=0.0)
    o = orc.iou_paired(d["p1"], d["p2"], d["c1"], d["c2"])
    r = W.rng_for(99)
    for k in range(40):
        n1, n2 = int(d["c1"][k]), int(d["c2"][k])
        P = d["p1"][k, :n1].astype(np.float64)
        Q = d["p2"][k, :n2].astype(np.float64)
        lo = np.minimum(P.min(0), Q.min(0))
        hi = np.maximum(P.max(0), Q.max(0))
        N = 400_000
        pts = lo + (hi - lo) * r.uniform(size=(N, 2))

        def inside(poly, x):
            ok = np.ones(len(x), bool)
            for j in range(len(poly)):
                a, b = poly[j], poly[(j + 1) % len(poly)]
                ok &= (b[0] - a[0]) * (x[:, 1] - a[1]) - (b[1] - a[1]) * (x[:, 0] - a[0]) >= 0
            return ok

        frac = (inside(P, pts) & inside(Q, pts)).mean()
        box = np.prod(hi - lo)
        est = frac * box
        sigma = box * math.sqrt(max(frac * (1 - frac), 1.0 / N) / N)
        assert abs(est - o["areas"][k, 0]) <= 4 * sigma + 1e-12, k


# --------------------------------------------------------------- gradients


def _fd_check(orc, P, Q, K, h_rel=1e-6):
    iou, ai, a1, a2, nx, code, dg, st = orc.iou_pair_f64(P, Q, K)
    g1, g2 = orc.iou_backward_pair_f64(P, Q, 1.0, nx, code, K)
    L = max(np.abs(P - P[0]).max(), np.abs(Q - P[0]).max())
    h = h_rel * L
    num1 = np.zeros_like(P)
    num2 = np.zeros_like(Q)
    for which, arr, num in ((0, P, num1), (1, Q, num2)):
        for v in range(arr.shape[0]):
            for c in range(2):
                vals = []
                for sgn in (1, -1):
                    A = P.copy()
                    B = Q.copy()
                    (A if which == 0 else B)[v, c] += sgn * h
                    r = orc.iou_pair_f64(A, B, K)
                    if r[4] != nx or list(r[5]) != list(code):
                        return None  # flags change within +-h: not differentiable here
                    vals.append(r[0])
                num[v, c] = (vals[0] - vals[1]) / (2 * h)
    return (g1, g2), (num1, num2)


@pytest.mark.parametrize("K", [4, 8])
def test_finite_differences(orc, K):
    """Oracle backward = central finite differences of the oracle forward (FP64)."""
    if K == 4:
        d = W.paired_rect_4096(seed=9, n=200)
        pairs = [(d["p1"][k].astype(np.float64), d["p2"][k].astype(np.float64)) for k in range(200)]
    else:
        d = W.convex_pairs_4m(seed=9, n=200, degenerate_frac=0.0)
        pairs = [(d["p1"][k, :d["c1"][k]].astype(np.float64), d["p2"][k, :d["c2"][k]].astype(np.float64))
                 for k in range(200)]
    checked = 0
    for P, Q in pairs:
        r = orc.iou_pair_f64(P, Q, K)
        if r[6] or r[4] == 0:
            continue
        res = _fd_check(orc, P, Q, K)
        if res is None:
            continue
        (g1, g2), (n1, n2) = res
        scale = max(np.abs(n1).max(), np.abs(n2).max(), 1e-6)
        err = max(np.abs(g1 - n1).max(), np.abs(g2 - n2).max()) / scale
        assert err <= 1e-6, err
        checked += 1
    assert checked >= 60


def test_gradient_invariants(orc):
    """IoU is invariant under translation, rotation and scaling of both
    polygons, so sum g = 0, sum cross(v, g) = 0 and sum v . g = 0."""
    d = W.convex_pairs_4m(seed=10, n=2000, degenerate_frac=0.0)
    K = 8
    o = orc.iou_paired(d["p1"], d["p2"], d["c1"], d["c2"])
    g1, g2 = orc.iou_backward_paired(d["p1"], d["p2"], np.ones(2000), o["nx"], o["xflags"], d["c1"], d["c2"])
    checked = 0
    for k in range(2000):
        if o["nx"][k] == 0:
            continue
        n1, n2 = int(d["c1"][k]), int(d["c2"][k])
        V = np.concatenate([d["p1"][k, :n1], d["p2"][k, :n2]]).astype(np.float64)
        G = np.concatenate([g1[k, :n1], g2[k, :n2]])
        # padded slots receive no gradient
        assert (g1[k, n1:] == 0).all() and (g2[k, n2:] == 0).all()
        V = V - V.mean(0)
        gn = np.abs(G).max()
        L = np.abs(V).max()
        tol = 1e-10 * max(gn, 1e-12) * max(L, 1.0)
        assert np.abs(G.sum(0)).max() <= tol
        assert abs((V[:, 0] * G[:, 1] - V[:, 1] * G[:, 0]).sum()) <= tol * L
        assert abs((V * G).sum()) <= tol * L
        checked += 1
    assert checked > 500
    assert K == 8


def test_empty_and_bad_counts(orc):
    """n = 0 is a no-op; counts outside [3, K] report ST_BAD_COUNT and IoU 0."""
    z = np.zeros((0, 4, 2), np.float32)
    o = orc.iou_paired(z, z)
    assert o["iou"].shape == (0,)
    d = W.paired_rect_4096(seed=1, n=4)
    o = orc.iou_paired(d["p1"], d["p2"], np.array([4, 2, 5, 4], np.uint8), None)
    assert o["status"] & orc.ST_BAD_COUNT
    assert o["iou"][1] == 0 and o["iou"][2] == 0 and o["iou"][0] > 0


def test_constructed_degenerate_kinds(orc):
    """Constructed degenerate partners: identical -> 1, shared edge and
    touching vertex -> 0, collinear offset -> the IoU of a translated copy."""
    d = W.convex_pairs_4m(seed=2, n=4000, degenerate_frac=0.2)
    o = orc.iou_paired(d["p1"], d["p2"], d["c1"], d["c2"])
    kind = d["kind"]
    assert np.abs(o["iou"][kind == 1] - 1).max() <= 1e-12
    assert np.abs(o["iou"][kind == 2]).max() <= 1e-12
    assert np.abs(o["iou"][kind == 3]).max() <= 1e-12
    assert (o["degen"][kind > 0] == 1).all()
    # collinear offset: compare with the exact rational clip
    for k in np.nonzero(kind == 4)[0][:30]:
        n1 = int(d["c1"][k])
        P = [tuple(v) for v in d["p1"][k, :n1]]
        Q = [tuple(v) for v in d["p2"][k, :n1]]
        inter = exact_clip.clip(P, Q)
        ai = float(exact_clip.area(inter)) if len(inter) >= 3 else 0.0
        assert abs(o["areas"][k, 0] - ai) <= 1e-12 * max(1.0, ai)


# ------------------------------------------- near-degenerate classifier
#
# The classifier decides where bit-exact nx / xflags are waived, so it is
# pinned on both sides: each family below places one quantity of the
# definition (with L the largest |coordinate| about P1's vertex 0) at a chosen
# multiple of its threshold by construction, with every other quantity of the
# pair far from its own threshold.  At 0.7 of the threshold the pair must be
# flagged and at 1.4 it must not be; a threshold taken 10 times too large, an
# L taken about the origin (the 70 m offset) or a criterion missing its
# guard flags a pair it must not, and a criterion left out misses one.


def _orient_family(ratio, off=0.0):
    """(i): the bottom vertex of a diamond sits 2 delta above the line of the
    square's top edge (length 2), so its orientation is 2 delta; L = 3.4 +
    delta.  delta solves 2 delta = ratio * 1e-5 L^2."""
    delta = 0.0
    for _ in range(4):
        delta = ratio * 1e-5 * (3.4 + delta) ** 2 / 2
    P = np.array([(0, 0), (2, 0), (2, 2), (0, 2)], np.float64) + off
    Q = np.array([(1, 2 + delta), (1.7, 2.7 + delta), (1, 3.4 + delta), (0.3, 2.7 + delta)], np.float64) + off
    P, Q = P.astype(np.float32), Q.astype(np.float32)
    # the construction's quantity from the rounded inputs: the orientation of
    # Q[0] against the top edge (2,2) -> (0,2) is 2 (y(Q[0]) - y(P[2]))
    d = 2.0 * (float(Q[0, 1]) - float(P[2, 1]))
    L = float(np.abs(np.concatenate([P, Q]).astype(np.float64) - P[0].astype(np.float64)).max())
    return P, Q, d / (1e-5 * L * L)


def _crossing_family(ratio):
    """(ii): an edge of Q (direction (1, 2), 8 long times the sine) crosses the
    square's bottom edge at x = 2 eps, i.e. at t = eps; the orientation of the
    square's vertex 0 against that edge is 7.2 eps, above 1e-5 L^2 = 4e-5 for
    eps >= 0.6e-5.  eps = ratio * 1e-5."""
    eps = ratio * 1e-5
    P = np.array([(0, 0), (2, 0), (2, 2), (0, 2)], np.float32)
    Q = np.array([(2 * eps - 0.9, -1.8), (2 * eps + 0.9, 1.8), (-1.2, 1.9), (-1.9, -0.5)], np.float32)
    c0, c1 = Q[0].astype(np.float64), Q[1].astype(np.float64)
    x = c0[0] + (0.0 - c0[1]) / (c1[1] - c0[1]) * (c1[0] - c0[0])  # where Q's edge 0 meets y = 0
    return P, Q, (x / 2.0) / 1e-5


def _parallel_family(ratio, apart=False):
    """(iii): Q's edge 0 runs from (3, 1.5 + eta) to (1.5, 0), against P's edge
    0 from (0, 0) to (2, 2): |cross(r, s)| = 2 eta with |r||s| = 6 (about), so
    eta = ratio * 3e-5.  The two lines are 1.06 apart, so no orientation is
    small.  apart=True moves Q by (1.5, -1.5): the edges' bounding boxes no
    longer overlap."""
    eta = ratio * 3e-5
    P = np.array([(0, 0), (2, 2), (0.9, 2.6), (-0.6, 1.5)], np.float32)
    Q = np.array([(3, 1.5 + eta), (1.5, 0), (2.5, -1), (3.5, 0.5)], np.float64)
    if apart:
        Q = Q + np.array([1.5, -1.5])
    Q = Q.astype(np.float32)
    r = (P[1] - P[0]).astype(np.float64)
    s = (Q[1] - Q[0]).astype(np.float64)
    return P, Q, abs(r[0] * s[1] - r[1] * s[0]) / (1e-5 * np.hypot(*r) * np.hypot(*s))


def _degen_flag(orc, P, Q):
    return int(orc.iou_paired(P[None], Q[None])["degen"][0])


@pytest.mark.parametrize("off", [0.0, 70.0], ids=["local", "offset70m"])
def test_degenerate_orientation_threshold(orc, off):
    lo, hi = _orient_family(0.7, off), _orient_family(1.4, off)
    assert 0.5 < lo[2] < 0.9 and 1.2 < hi[2] < 1.7, (lo[2], hi[2])
    assert _degen_flag(orc, lo[0], lo[1]) == 1
    assert _degen_flag(orc, hi[0], hi[1]) == 0


def test_degenerate_crossing_parameter_threshold(orc):
    lo, hi = _crossing_family(0.7), _crossing_family(1.4)
    assert 0.6 < lo[2] < 0.8 and 1.3 < hi[2] < 1.5, (lo[2], hi[2])
    o = orc.iou_paired(np.stack([lo[0], hi[0]]), np.stack([lo[1], hi[1]]))
    assert list(o["degen"]) == [1, 0]
    # the crossing is a real one: the intersection has a crossing code on
    # P's edge 0 with Q's edge 0
    assert 0x80 in list(o["xflags"][1])


def test_degenerate_parallel_threshold(orc):
    lo, hi = _parallel_family(0.7), _parallel_family(1.4)
    assert 0.6 < lo[2] < 0.8 and 1.3 < hi[2] < 1.5, (lo[2], hi[2])
    assert _degen_flag(orc, lo[0], lo[1]) == 1
    assert _degen_flag(orc, hi[0], hi[1]) == 0
    # exactly parallel edges whose bounding boxes do not overlap are not a
    # near-degenerate configuration
    P, Q, ratio = _parallel_family(0.0, apart=True)
    assert ratio == 0.0
    assert _degen_flag(orc, P, Q) == 0


def test_degenerate_rate_on_loss_workload(orc):
    """The IoU-loss pairs are generic: the classifier flags a small fraction
    (0.13% measured), so the waiver of bit-exactness stays rare."""
    d = W.loss_pairs_1m(seed=0, n=200_000)
    o = orc.iou_paired(d["p1"], d["p2"], threads=8)
    assert o["degen"].mean() < 0.005


def test_gradient_magnitude_bound(orc):
    """|dIoU/dv| <= 3 * 2 sqrt(2) L / U for every vertex (the IoU's derivative
    through the three areas, each moved by at most the pair's diameter per
    unit of vertex motion): holds on every pair, near-degenerate ones
    included, and is the bound the GPU tests apply to pairs the parity bar
    waives."""
    from .gpu_helpers import check_flagged_grads

    d = W.convex_pairs_4m(seed=5, n=20_000, degenerate_frac=0.2)
    ref = orc.iou_paired(d["p1"], d["p2"], d["c1"], d["c2"], threads=8)
    g1, g2 = orc.iou_backward_paired(d["p1"], d["p2"], np.ones(20_000), ref["nx"], ref["xflags"], d["c1"], d["c2"],
                                     threads=8)
    check_flagged_grads(g1, g2, d["p1"], d["p2"], d["c1"], d["c2"], ref, np.ones(20_000, bool), label="oracle")
