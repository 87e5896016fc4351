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
