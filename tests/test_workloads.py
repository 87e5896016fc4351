"""The seeded input generators follow their stated recipes (shapes, ranges,
orientation, determinism, ragged offsets, the constructed degenerate kinds).
They hold none of the method's arithmetic; these checks use only numpy."""
import numpy as np
import pytest

from paper_2011_11134_gb300 import workloads as W


def _signed_area(p, cnt=None):
    """Twice the shoelace area of each polygon's first cnt vertices (float64)."""
    p = p.astype(np.float64)
    n, K = p.shape[:2]
    cnt = np.full(n, K) if cnt is None else cnt.astype(int)
    out = np.zeros(n)
    for k in range(K):
        nxt = np.where(k + 1 < cnt, k + 1, 0)
        on = k < cnt
        a = p[np.arange(n), k]
        b = p[np.arange(n), nxt]
        out += np.where(on, a[:, 0] * b[:, 1] - a[:, 1] * b[:, 0], 0.0)
    return out


def _sides(p):
    """Side lengths of quadrilaterals [n, 4, 2] (float64): [n, 4]."""
    q = p.astype(np.float64)
    return np.linalg.norm(np.roll(q, -1, axis=1) - q, axis=2)


def test_boxes_to_polygons_corners():
    p = W.boxes_to_polygons([1.0], [2.0], [4.0], [2.0], [np.pi / 2])
    # w = 4 along the rotated x axis (now +y), h = 2 along -x; CCW from (-w/2, -h/2)
    ref = np.array([[[2.0, 0.0], [2.0, 4.0], [0.0, 4.0], [0.0, 0.0]]])
    assert p.dtype == np.float32 and p.shape == (1, 4, 2)
    assert np.allclose(p, ref, atol=1e-6)


@pytest.mark.parametrize("gen", [W.paired_rect_4096, W.loss_pairs_1m])
def test_paired_rectangles(gen):
    d = gen(seed=3, n=5000)
    e = gen(seed=3, n=5000)
    assert np.array_equal(d["p1"], e["p1"]) and np.array_equal(d["p2"], e["p2"])  # seeded
    assert not np.array_equal(d["p1"], gen(seed=4, n=5000)["p1"])
    for p in (d["p1"], d["p2"]):
        assert p.shape == (5000, 4, 2) and p.dtype == np.float32
        assert (_signed_area(p) > 0).all()  # counter-clockwise
        s = _sides(p)
        assert np.allclose(s[:, 0], s[:, 2], rtol=1e-5) and np.allclose(s[:, 1], s[:, 3], rtol=1e-5)
    assert (d["grad"] == 1).all()


def test_rect_4096_ranges():
    d = W.paired_rect_4096(seed=0)
    s = _sides(d["p1"])
    assert s.min() >= 0.5 - 1e-5 and s.max() <= 4.0 + 1e-5  # w, h ~ U[0.5, 4]
    c = d["p1"].astype(np.float64).mean(1)
    assert c.min() >= -1e-5 and c.max() <= 10.0 + 1e-5  # centres ~ U[0, 10]^2
    s2 = _sides(d["p2"])
    assert s2.min() >= 0.35 - 1e-5 and s2.max() <= 5.2 + 1e-5  # scaled by U[0.7, 1.3]


def test_bev_boxes_ranges():
    d = W.pairwise_bev_2000(seed=1)
    for p in (d["a"], d["b"]):
        assert p.shape == (2000, 4, 2)
        assert (_signed_area(p) > 0).all()
        s = _sides(p)
        length, width = s[:, 0], s[:, 1]  # length along the box's own x axis
        assert length.min() >= 3.5 - 1e-4 and length.max() <= 5.0 + 1e-4
        assert width.min() >= 1.5 - 1e-4 and width.max() <= 2.2 + 1e-4
    # 40 clusters in a 70 m plane, sigma 3 m: centres stay near it
    c = d["a"].astype(np.float64).mean(1)
    assert c.min() > -25 and c.max() < 95


def test_ragged_scenes_offsets():
    d = W.ragged_scenes_64(seed=2)
    Ns = np.diff(d["a_off"])
    Ms = np.diff(d["b_off"])
    assert len(Ns) == 64 and d["a_off"][0] == 0 and d["b_off"][0] == 0 and d["out_off"][0] == 0
    assert Ns.min() >= 50 and Ns.max() <= 3000 and Ms.min() >= 5 and Ms.max() <= 200
    assert np.array_equal(np.diff(d["out_off"]), Ns * Ms)
    assert d["a"].shape == (d["a_off"][-1], 4, 2) and d["b"].shape == (d["b_off"][-1], 4, 2)


def test_loss3d_extents():
    d = W.loss3d_pairs_1m(seed=5, n=4000)
    z1, z2 = d["z1"].astype(np.float64), d["z2"].astype(np.float64)
    assert z1.shape == (4000, 2) and z2.shape == (4000, 2)
    assert z2[:, 0].min() >= -1 and z2[:, 0].max() <= 1
    assert z2[:, 1].min() >= 1.4 - 1e-6 and z2[:, 1].max() <= 1.8 + 1e-6
    assert (z1[:, 1] > 0).all()
    assert np.array_equal(d["p1"], W.loss_pairs_1m(seed=5, n=4000)["p1"])  # same bird's-eye view


def test_convex_pairs_recipe():
    n = 4000
    d = W.convex_pairs_4m(seed=6, n=n)
    p1, c1, p2, c2, kind = d["p1"], d["c1"], d["p2"], d["c2"], d["kind"]
    assert p1.shape == (n, 8, 2) and c1.dtype == np.uint8
    assert c1.min() >= 3 and c1.max() <= 8 and c2.min() >= 3 and c2.max() <= 8
    assert (_signed_area(p1, c1) > 0).all() and (_signed_area(p2, c2) > 0).all()
    # 5% constructed near-degenerate pairs, split equally over the four kinds
    counts = np.bincount(kind, minlength=5)
    assert counts[1:].sum() == round(0.05 * n) and counts[1:].max() - counts[1:].min() <= 1
    for k in np.flatnonzero(kind == 1)[:50]:  # identical partner
        assert np.array_equal(p1[k, : c1[k]], p2[k, : c2[k]])
    for k in np.flatnonzero(kind == 2)[:50]:  # shared edge: two vertices copied bit-exactly
        a = {tuple(v) for v in p1[k, : c1[k]].tolist()}
        assert sum(tuple(v) in a for v in p2[k, : c2[k]].tolist()) >= 2
    for k in np.flatnonzero(kind == 3)[:50]:  # touching vertex: exactly one shared vertex
        a = {tuple(v) for v in p1[k, : c1[k]].tolist()}
        assert sum(tuple(v) in a for v in p2[k, : c2[k]].tolist()) == 1
    for k in np.flatnonzero(kind == 4)[:50]:  # shifted copy: same shape, moved off the lattice
        q1, q2 = p1[k, : c1[k]].astype(np.float64), p2[k, : c2[k]].astype(np.float64)
        assert c1[k] == c2[k]
        assert np.allclose((q2 - q1) - (q2 - q1).mean(0), 0.0, atol=1e-5)


def test_convex_pairs_k4_counts():
    d = W.convex_pairs_4m(seed=7, n=2000, K=4, degenerate_frac=0.0)
    assert d["p1"].shape == (2000, 4, 2)
    assert set(np.unique(d["c1"])) <= {3, 4} and (d["kind"] == 0).all()
