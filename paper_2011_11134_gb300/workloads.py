"""Seeded synthetic workloads for convex-polygon IoU (shared by tests, smoke and bench).

This module only builds inputs: boxes -> counter-clockwise corner polygons,
convex hulls of random points, constructed degenerate partners.  It holds none
of the intersection / area / IoU arithmetic, so the CUDA path and the CPU
oracle can both consume its arrays without sharing any of the method.

The paper's case study (Sec. IV-A, rotated 2D IoU loss on rotated bounding
boxes) names no public dataset; these generators stand in for it.

All randomness comes from ``numpy.random.Generator(PCG64(seed))``.  Polygons
are float32 arrays [n, K, 2] (x, y interleaved, counter-clockwise); general
polygons also carry uint8 vertex counts.
"""
from __future__ import annotations

import os

import numpy as np


def rng_for(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def boxes_to_polygons(cx, cy, w, h, theta) -> np.ndarray:
    """Rotated boxes -> float32 [n, 4, 2] corners in counter-clockwise order.

    Local corners (-w/2,-h/2), (w/2,-h/2), (w/2,h/2), (-w/2,h/2) are rotated by
    theta and translated to (cx, cy); computed in float64, stored as float32."""
    cx, cy, w, h, theta = (np.asarray(v, dtype=np.float64) for v in (cx, cy, w, h, theta))
    lx = np.stack([-w / 2, w / 2, w / 2, -w / 2], axis=-1)
    ly = np.stack([-h / 2, -h / 2, h / 2, h / 2], axis=-1)
    c, s = np.cos(theta)[..., None], np.sin(theta)[..., None]
    x = cx[..., None] + c * lx - s * ly
    y = cy[..., None] + s * lx + c * ly
    return np.stack([x, y], axis=-1).astype(np.float32)


# ----------------------------------------------------------------- configs


def paired_rect_4096(seed: int = 0, n: int = 4096):
    """Paired rotated rectangles, K=4 (4096 pairs by default).

    Box a: center ~ U[0,10]^2, w,h ~ U[0.5,4], theta ~ U[-pi,pi).
    Box b: a's center + N(0,1)^2, w,h scaled by U[0.7,1.3], theta + N(0,0.3).
    Upstream gradient dL/dIoU = 1."""
    r = rng_for(seed)
    c = r.uniform(0.0, 10.0, size=(n, 2))
    wh = r.uniform(0.5, 4.0, size=(n, 2))
    th = r.uniform(-np.pi, np.pi, size=n)
    c2 = c + r.normal(0.0, 1.0, size=(n, 2))
    wh2 = wh * r.uniform(0.7, 1.3, size=(n, 2))
    th2 = th + r.normal(0.0, 0.3, size=n)
    p1 = boxes_to_polygons(c[:, 0], c[:, 1], wh[:, 0], wh[:, 1], th)
    p2 = boxes_to_polygons(c2[:, 0], c2[:, 1], wh2[:, 0], wh2[:, 1], th2)
    return dict(p1=p1, p2=p2, grad=np.ones(n, np.float32))


def _bev_boxes(r: np.random.Generator, centers: np.ndarray, n: int) -> np.ndarray:
    k = r.integers(0, centers.shape[0], size=n)
    c = centers[k] + r.normal(0.0, 3.0, size=(n, 2))
    w = r.uniform(1.5, 2.2, size=n)
    length = r.uniform(3.5, 5.0, size=n)
    th = r.uniform(-np.pi, np.pi, size=n)
    return boxes_to_polygons(c[:, 0], c[:, 1], length, w, th)


def bev_clusters(r: np.random.Generator, n_clusters: int = 40, extent: float = 70.0) -> np.ndarray:
    return r.uniform(0.0, extent, size=(n_clusters, 2))


def pairwise_bev_2000(seed: int = 0, N: int = 2000, M: int = 2000):
    """Pairwise matrix workload: N x M car-like boxes in a 70 m x 70 m plane.

    40 cluster centers ~ U[0,70]^2; each box picks a cluster uniformly, center
    ~ N(cluster, 3^2 I), width ~ U[1.5,2.2], length ~ U[3.5,5], theta ~
    U[-pi,pi).  Both sets are drawn from the same clusters."""
    r = rng_for(seed)
    centers = bev_clusters(r)
    return dict(a=_bev_boxes(r, centers, N), b=_bev_boxes(r, centers, M))


def ragged_scenes_64(seed: int = 0, S: int = 64, n_range=(50, 3000), m_range=(5, 200)):
    """Ragged batch: S scenes, N_i ~ U{50..3000} boxes vs M_i ~ U{5..200}.

    Each scene has its own 40 clusters and boxes as in the pairwise workload.
    Returns packed a [sum N_i, 4, 2], b [sum M_i, 4, 2] and int64 offsets
    a_off, b_off, out_off (out_off[s+1]-out_off[s] = N_s M_s)."""
    r = rng_for(seed)
    Ns = r.integers(n_range[0], n_range[1] + 1, size=S)
    Ms = r.integers(m_range[0], m_range[1] + 1, size=S)
    a_list, b_list = [], []
    for s in range(S):
        centers = bev_clusters(r)
        a_list.append(_bev_boxes(r, centers, int(Ns[s])))
        b_list.append(_bev_boxes(r, centers, int(Ms[s])))
    a_off = np.zeros(S + 1, np.int64)
    b_off = np.zeros(S + 1, np.int64)
    out_off = np.zeros(S + 1, np.int64)
    a_off[1:] = np.cumsum(Ns)
    b_off[1:] = np.cumsum(Ms)
    out_off[1:] = np.cumsum(Ns.astype(np.int64) * Ms.astype(np.int64))
    return dict(a=np.concatenate(a_list), b=np.concatenate(b_list), a_off=a_off, b_off=b_off, out_off=out_off,
                N=Ns.astype(np.int64), M=Ms.astype(np.int64))


def loss_pairs_1m(seed: int = 0, n: int = 1_000_000):
    """IoU-loss pairs, K=4: target as in the 4096-pair workload; prediction =
    target + center N(0,0.5)^2, log w / log h + N(0,0.2), theta + N(0,0.2).

    Returns p1 = prediction, p2 = target, upstream grad = 1."""
    r = rng_for(seed)
    c = r.uniform(0.0, 10.0, size=(n, 2))
    wh = r.uniform(0.5, 4.0, size=(n, 2))
    th = r.uniform(-np.pi, np.pi, size=n)
    cp = c + r.normal(0.0, 0.5, size=(n, 2))
    whp = np.exp(np.log(wh) + r.normal(0.0, 0.2, size=(n, 2)))
    thp = th + r.normal(0.0, 0.2, size=n)
    target = boxes_to_polygons(c[:, 0], c[:, 1], wh[:, 0], wh[:, 1], th)
    pred = boxes_to_polygons(cp[:, 0], cp[:, 1], whp[:, 0], whp[:, 1], thp)
    return dict(p1=pred, p2=target, grad=np.ones(n, np.float32))


def loss3d_pairs_1m(seed: int = 0, n: int = 1_000_000):
    """3D IoU-loss pairs (rotated boxes with a vertical extent), K=4: the
    bird's-eye view as in the IoU-loss pairs; target extent z ~ U[-1, 1],
    h ~ U[1.4, 1.8]; prediction z + N(0, 0.2), h * exp(N(0, 0.1)).

    Returns p1, z1 = prediction, p2, z2 = target (z = [n, 2] = (z_center,
    height)), upstream grad = 1."""
    d = loss_pairs_1m(seed, n)
    r = rng_for(seed + 7919)
    z = r.uniform(-1.0, 1.0, size=n)
    h = r.uniform(1.4, 1.8, size=n)
    zp = z + r.normal(0.0, 0.2, size=n)
    hp = h * np.exp(r.normal(0.0, 0.1, size=n))
    d["z1"] = np.stack([zp, hp], 1).astype(np.float32)
    d["z2"] = np.stack([z, h], 1).astype(np.float32)
    return d


# ----------------------------------------------------- general convex polygons


def _strictly_convex_ccw(poly: np.ndarray, cnt: np.ndarray) -> np.ndarray:
    """True where every consecutive vertex triple (in float64 on the stored
    float32 values) turns strictly left, i.e. a valid convex CCW input (row
    chunks on a thread pool for large inputs)."""
    n = poly.shape[0]
    chunk = 1 << 16
    if n > chunk:
        from concurrent.futures import ThreadPoolExecutor

        spans = [(s, min(n, s + chunk)) for s in range(0, n, chunk)]
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            return np.concatenate(list(ex.map(lambda se: _strictly_convex_ccw(poly[se[0]:se[1]], cnt[se[0]:se[1]]),
                                              spans)))
    n, K, _ = poly.shape
    p = poly.astype(np.float64)
    ok = np.ones(n, bool)
    for v in range(K):
        valid = v < cnt
        i0 = v
        i1 = np.where(v + 1 < cnt, v + 1, 0)
        i2 = np.where(v + 2 < cnt, v + 2, v + 2 - cnt)
        i2 = np.clip(i2, 0, K - 1)
        a = p[np.arange(n), i0]
        b = p[np.arange(n), i1]
        c = p[np.arange(n), i2]
        t = (b[:, 0] - a[:, 0]) * (c[:, 1] - b[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - b[:, 0])
        ok &= ~valid | (t > 0)
    return ok


def _hull_points(pts: np.ndarray, m: np.ndarray, centers: np.ndarray, K: int):
    """Convex hull (counter-clockwise, padded with vertex 0) of the first m
    points of each row of pts (relative to the row's center)."""
    n = pts.shape[0]
    valid = np.arange(K)[None, :] < m[:, None]
    # sort valid points by angle about their mean (an interior point)
    mean = (pts * valid[..., None]).sum(1) / m[:, None]
    d = pts - mean[:, None, :]
    a = np.arctan2(d[..., 1], d[..., 0])
    a = np.where(valid, a, np.inf)
    order = np.argsort(a, axis=1)
    pts = np.take_along_axis(pts, order[..., None], axis=1)
    alive = np.take_along_axis(valid, order, axis=1)
    # drop reflex vertices until none is left (each dropped point lies inside
    # the triangle mean-prev-next, hence inside the hull, so dropping all of
    # them in one sweep is safe)
    cols = np.arange(K)[None, :]
    X, Y = np.ascontiguousarray(pts[..., 0]), np.ascontiguousarray(pts[..., 1])
    for _ in range(K):
        # cyclic previous / next alive point of every position
        pm = np.maximum.accumulate(np.where(alive, cols, -1), axis=1)  # last alive at or before i
        prv = np.concatenate([np.full((n, 1), -1), pm[:, :-1]], 1)
        prv = np.where(prv < 0, pm[:, -1:], prv)
        nm = np.minimum.accumulate(np.where(alive, cols, K)[:, ::-1], axis=1)[:, ::-1]  # first alive at or after i
        nxt = np.concatenate([nm[:, 1:], np.full((n, 1), K)], 1)
        nxt = np.where(nxt >= K, nm[:, :1], nxt)
        Xp, Yp = np.take_along_axis(X, prv, 1), np.take_along_axis(Y, prv, 1)
        Xn, Yn = np.take_along_axis(X, nxt, 1), np.take_along_axis(Y, nxt, 1)
        t = (X - Xp) * (Yn - Y) - (Y - Yp) * (Xn - X)
        drop = alive & (t <= 0)
        if not drop.any():
            break
        alive &= ~drop
    cnt = alive.sum(1)
    order = np.argsort(~alive, axis=1, kind="stable")
    pts = np.take_along_axis(pts, order[..., None], axis=1)
    pts = pts + centers[:, None, :]
    first = pts[:, :1, :]
    pad = np.arange(K)[None, :, None] >= cnt[:, None, None]
    pts = np.where(pad, first, pts)
    return pts.astype(np.float32), cnt.astype(np.uint8)


def _hulls(r: np.random.Generator, centers: np.ndarray, K: int):
    """Convex hull of 3..K points uniform in a disc (radius ~ U[0.5,3]) around
    each center; returns float32 [n, K, 2] padded with vertex 0 and counts.
    The random draws come first, in one sequence; the hulls are then built in
    row chunks on a thread pool (the result does not depend on the chunks)."""
    n = centers.shape[0]
    m = r.integers(3, K + 1, size=n)
    rad = r.uniform(0.5, 3.0, size=n)
    ang = r.uniform(-np.pi, np.pi, size=(n, K))
    rr = rad[:, None] * np.sqrt(r.uniform(0.0, 1.0, size=(n, K)))
    pts = np.stack([rr * np.cos(ang), rr * np.sin(ang)], axis=-1)  # relative to center
    chunk = 1 << 16
    if n <= chunk:
        return _hull_points(pts, m, centers, K)
    from concurrent.futures import ThreadPoolExecutor

    spans = [(s, min(n, s + chunk)) for s in range(0, n, chunk)]
    with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
        parts = list(ex.map(lambda se: _hull_points(pts[se[0]:se[1]], m[se[0]:se[1]], centers[se[0]:se[1]], K),
                            spans))
    return np.concatenate([p for p, _ in parts]), np.concatenate([c for _, c in parts])


def convex_pairs_4m(seed: int = 0, n: int = 4_000_000, K: int = 8, degenerate_frac: float = 0.05):
    """General convex polygons (K=8, counts 3..8), paired.

    P1: convex hull of 3..8 points uniform in a disc of radius ~U[0.5,3],
    disc center ~ U[0,10]^2.  P2: the same recipe about P1's center +
    N(0,1)^2.  Hulls that are not strictly convex after float32 rounding are
    redrawn.  A fraction ``degenerate_frac`` of pairs is replaced by
    constructed near-degenerate partners, split equally over
      1 identical (P2 = P1),
      2 shared edge (P2 = P1 reflected across one of its edges, the edge's
        endpoints copied bit-exactly, order reversed to stay CCW),
      3 single touching vertex (P2 = P1 point-reflected through one vertex:
        interiors are disjoint by convexity, the vertex is shared exactly),
      4 collinear edge offset (P2 = P1 shifted along one edge by U[-1/4,1/4]
        of its length and 1e-6 along its normal).
    Returns p1, c1, p2, c2 and kind (uint8: 0 generic, 1..4 as above)."""
    r = rng_for(seed)
    centers = r.uniform(0.0, 10.0, size=(n, 2))
    p1, c1 = _hulls(r, centers, K)
    p2, c2 = _hulls(r, centers + r.normal(0.0, 1.0, size=(n, 2)), K)
    for _ in range(20):
        bad1 = ~_strictly_convex_ccw(p1, c1) | (c1 < 3)
        bad2 = ~_strictly_convex_ccw(p2, c2) | (c2 < 3)
        if not (bad1.any() or bad2.any()):
            break
        if bad1.any():
            q, qc = _hulls(r, centers[bad1], K)
            p1[bad1], c1[bad1] = q, qc
        if bad2.any():
            q, qc = _hulls(r, centers[bad2] + r.normal(0.0, 1.0, size=(int(bad2.sum()), 2)), K)
            p2[bad2], c2[bad2] = q, qc
    kind = np.zeros(n, np.uint8)
    nd = int(round(degenerate_frac * n))
    if nd:
        idx = r.choice(n, size=nd, replace=False)
        kinds = (np.arange(nd) % 4 + 1).astype(np.uint8)
        kind[idx] = kinds
        sel_v = r.integers(0, 1 << 30, size=nd)
        shift = r.uniform(-0.25, 0.25, size=nd)
        sign = np.where(r.uniform(size=nd) < 0.5, -1.0, 1.0)
        m = c1[idx].astype(np.int64)
        e = sel_v % m
        e1 = (e + 1) % m
        rows = np.arange(nd)
        P = p1[idx].astype(np.float64)  # [nd, K, 2]; slots >= m repeat vertex 0
        live = np.arange(K)[None, :] < m[:, None]
        a, b = P[rows, e], P[rows, e1]
        q = np.empty((nd, K, 2), np.float32)
        # 1 identical
        q1 = p1[idx]
        # 2 reflection across edge e, its endpoints copied exactly, order reversed
        d = (b - a) / np.linalg.norm(b - a, axis=1, keepdims=True)
        rel = P - a[:, None, :]
        proj = rel[..., 0] * d[:, None, 0] + rel[..., 1] * d[:, None, 1]
        Q2 = (a[:, None, :] + 2 * proj[..., None] * d[:, None, :] - rel).astype(np.float32)
        Q2[rows, e] = p1[idx][rows, e]
        Q2[rows, e1] = p1[idx][rows, e1]
        rev = np.where(live, m[:, None] - 1 - np.arange(K)[None, :], 0)  # reversed order of the m live slots
        Q2 = np.take_along_axis(Q2, rev[..., None], axis=1)
        # 3 point reflection through vertex e, which is kept exactly
        Q3 = (2 * a[:, None, :] - P).astype(np.float32)
        Q3[rows, e] = p1[idx][rows, e]
        # 4 shifted along edge e by U[-1/4, 1/4] of its length and 1e-6 along its normal
        Le = np.linalg.norm(b - a, axis=1)
        nrm = np.stack([-d[:, 1], d[:, 0]], 1)
        Q4 = (P + (shift * Le)[:, None, None] * d[:, None, :] + (sign * 1e-6)[:, None, None] * nrm[:, None, :]).astype(
            np.float32)
        kk = kinds[:, None, None]
        q = np.where(kk == 1, q1, np.where(kk == 2, Q2, np.where(kk == 3, Q3, Q4)))
        q = np.where(live[..., None], q, q[:, :1, :])  # pad with vertex 0
        p2[idx] = q
        c2[idx] = c1[idx]
    return dict(p1=p1, c1=c1, p2=p2, c2=c2, kind=kind)
