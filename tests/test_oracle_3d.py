"""Pins for the oracle's 3D IoU (bird's-eye polygon x vertical extent) and
its gradient: the cuboid closed form, special cases, symmetry, and central
differences of the double-precision forward."""
import numpy as np

from paper_2011_11134_gb300 import workloads as W


def _aabb(c, wh):
    lo, hi = c - wh / 2, c + wh / 2
    return np.stack([lo, [hi[0], lo[1]], hi, [lo[0], hi[1]]]).astype(np.float32)


def test_axis_aligned_cuboids_closed_form(orc):
    r = np.random.default_rng(31)
    n = 300
    c1 = r.uniform(0, 4, (n, 3)).astype(np.float32)
    c2 = (c1 + r.normal(0, 0.8, (n, 3))).astype(np.float32)
    s1 = r.uniform(0.5, 2.5, (n, 3)).astype(np.float32)
    s2 = r.uniform(0.5, 2.5, (n, 3)).astype(np.float32)
    p1 = np.stack([_aabb(c1[k, :2], s1[k, :2]) for k in range(n)])
    p2 = np.stack([_aabb(c2[k, :2], s2[k, :2]) for k in range(n)])
    z1 = np.stack([c1[:, 2], s1[:, 2]], 1)
    z2 = np.stack([c2[:, 2], s2[:, 2]], 1)
    f = orc.iou3d_paired(p1, p2, z1, z2)
    # exact corners in double from the float corners and extents
    P1, P2 = p1.astype(np.float64), p2.astype(np.float64)
    lo1, hi1 = P1.min(1), P1.max(1)
    lo2, hi2 = P2.min(1), P2.max(1)
    Z1, Z2 = z1.astype(np.float64), z2.astype(np.float64)
    zl1, zh1 = Z1[:, 0] - Z1[:, 1] / 2, Z1[:, 0] + Z1[:, 1] / 2
    zl2, zh2 = Z2[:, 0] - Z2[:, 1] / 2, Z2[:, 0] + Z2[:, 1] / 2
    ext = np.clip(np.minimum(hi1, hi2) - np.maximum(lo1, lo2), 0, None)
    ez = np.clip(np.minimum(zh1, zh2) - np.maximum(zl1, zl2), 0, None)
    inter = ext[:, 0] * ext[:, 1] * ez
    v1 = (hi1 - lo1).prod(1) * Z1[:, 1]
    v2 = (hi2 - lo2).prod(1) * Z2[:, 1]
    ref = inter / (v1 + v2 - inter)
    assert np.abs(f["iou"] - ref).max() <= 1e-12
    assert (ref > 0).sum() > 50 and (ref == 0).sum() > 10


def test_special_cases_and_symmetry(orc):
    d = W.paired_rect_4096(seed=32, n=200)
    r = np.random.default_rng(33)
    z1 = np.stack([r.uniform(-1, 1, 200), r.uniform(1, 2, 200)], 1).astype(np.float32)
    z2 = np.stack([r.uniform(-1, 1, 200), r.uniform(1, 2, 200)], 1).astype(np.float32)
    same = orc.iou3d_paired(d["p1"], d["p1"], z1, z1)
    assert np.abs(same["iou"] - 1.0).max() <= 1e-12
    # z-disjoint: 0 and zero gradients
    z_far = z2.copy()
    z_far[:, 0] += 10.0
    f = orc.iou3d_paired(d["p1"], d["p2"], z1, z_far)
    assert np.abs(f["iou"]).max() == 0.0
    g1, gz1, g2, gz2 = orc.iou3d_backward_paired(d["p1"], d["p2"], z1, z_far, np.ones(200), f["nx"], f["xflags"])
    assert max(np.abs(g).max() for g in (g1, gz1, g2, gz2)) == 0.0
    # same footprint, nested z-extents: IoU = short height / tall height
    zi = np.stack([z1[:, 0], z1[:, 1] * 0.5], 1).astype(np.float32)
    f = orc.iou3d_paired(d["p1"], d["p1"], z1, zi)
    assert np.abs(f["iou"] - zi[:, 1].astype(np.float64) / z1[:, 1]).max() <= 1e-12
    a = orc.iou3d_paired(d["p1"], d["p2"], z1, z2)["iou"]
    b = orc.iou3d_paired(d["p2"], d["p1"], z2, z1)["iou"]
    assert np.abs(a - b).max() <= 1e-12


def _iou3_f64(orc, P, Q, z1, z2):
    iou2, ai, a1, a2, nx, code, dg, st = orc.iou_pair_f64(P, Q, 4)
    lo1, hi1 = z1[0] - z1[1] / 2, z1[0] + z1[1] / 2
    lo2, hi2 = z2[0] - z2[1] / 2, z2[0] + z2[1] / 2
    ov = max(0.0, min(hi1, hi2) - max(lo1, lo2))
    inter = (ai if nx >= 3 else 0.0) * ov
    u = a1 * z1[1] + a2 * z2[1] - inter
    return (inter / u if u > 0 else 0.0), nx, list(code)


def test_gradient_finite_differences(orc):
    d = W.loss_pairs_1m(seed=34, n=40)
    r = np.random.default_rng(35)
    z1 = np.stack([r.uniform(-0.3, 0.3, 40), r.uniform(1.4, 1.8, 40)], 1).astype(np.float32)
    z2 = np.stack([z1[:, 0] + r.normal(0, 0.2, 40), z1[:, 1] * r.uniform(0.8, 1.2, 40)], 1).astype(np.float32)
    f = orc.iou3d_paired(d["p1"], d["p2"], z1, z2)
    g1, gz1, g2, gz2 = orc.iou3d_backward_paired(d["p1"], d["p2"], z1, z2, np.ones(40), f["nx"], f["xflags"])
    checked = 0
    for k in range(40):
        if f["degen"][k] or f["nx"][k] < 3 or f["ov"][k] <= 0:
            continue
        P, Q = d["p1"][k].astype(np.float64), d["p2"][k].astype(np.float64)
        Z1, Z2 = z1[k].astype(np.float64), z2[k].astype(np.float64)
        h = 1e-6 * max(np.abs(P - P[0]).max(), np.abs(Q - P[0]).max())
        base = _iou3_f64(orc, P, Q, Z1, Z2)
        num = [np.zeros((4, 2)), np.zeros(2), np.zeros((4, 2)), np.zeros(2)]
        ok = True
        for which, arr in enumerate((P, Z1, Q, Z2)):
            for idx in np.ndindex(arr.shape):
                vals = []
                for sg in (1, -1):
                    A = [P.copy(), Z1.copy(), Q.copy(), Z2.copy()]
                    A[which][idx] += sg * h
                    v, nxv, code = _iou3_f64(orc, A[0], A[2], A[1], A[3])
                    ok &= nxv == base[1] and code == base[2]
                    vals.append(v)
                num[which][idx] = (vals[0] - vals[1]) / (2 * h)
        if not ok:
            continue
        for G, N in zip((g1[k], gz1[k], g2[k], gz2[k]), num):
            assert np.abs(G - N).max() <= 1e-6 * max(np.abs(num[0]).max(), np.abs(num[1]).max(), 1e-9)
        checked += 1
    assert checked >= 30
