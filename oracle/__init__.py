"""FP64 CPU oracle for convex-polygon IoU and its gradient (DGAL, arXiv:2011.11134).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference arm are the only callers.  The product
path never imports this package.

The arithmetic lives in ``dgal_oracle.c`` (plain C, IEEE double, no FMA
contraction); this module builds it with gcc and wraps it with ctypes and
numpy.  Every function cites the passage of the paper it follows in the C
file.  Pins against independent results (closed forms, exact rational
clipping, point sampling, finite differences) are in ``tests/``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dgal_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# status bits (mirror of the C defines)
ST_BAD_COUNT = 1
ST_OVERFLOW = 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags, no contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            # DGAL_ORACLE_SO names another build of dgal_oracle.c (the mutation
            # test uses it to check that the pins catch planted mistakes).
            alt = os.environ.get("DGAL_ORACLE_SO")
            if not alt:
                build()
            lib = ctypes.CDLL(alt or _LIB)
            P = ctypes.c_void_p
            lib.oracle_iou_paired.argtypes = [ctypes.c_int64, ctypes.c_int, P, P, P, P, P, P, P, P, P]
            lib.oracle_iou_paired.restype = ctypes.c_int
            lib.oracle_iou_backward_paired.argtypes = [ctypes.c_int64, ctypes.c_int, P, P, P, P, P, P, P, P, P]
            lib.oracle_iou_backward_paired.restype = ctypes.c_int
            lib.oracle_area_backward_paired.argtypes = [ctypes.c_int64, ctypes.c_int] + [P] * 11
            lib.oracle_area_backward_paired.restype = ctypes.c_int
            lib.oracle_intersect_paired.argtypes = [ctypes.c_int64, ctypes.c_int, P, P, P, P, P, P, P]
            lib.oracle_intersect_paired.restype = ctypes.c_int
            lib.oracle_area.argtypes = [ctypes.c_int64, ctypes.c_int, P, P, P]
            lib.oracle_area.restype = ctypes.c_int
            lib.oracle_iou_pairwise.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int, P, P, P, P, P, P]
            lib.oracle_iou_pairwise.restype = ctypes.c_int
            lib.oracle_iou_pair_f64.argtypes = [ctypes.c_int, P, ctypes.c_int, P, ctypes.c_int, P, P, P, P]
            lib.oracle_iou_pair_f64.restype = ctypes.c_int
            lib.oracle_iou_backward_pair_f64.argtypes = [ctypes.c_int, P, ctypes.c_int, P, ctypes.c_int,
                                                         ctypes.c_double, ctypes.c_int, P, P, P]
            lib.oracle_iou_backward_pair_f64.restype = ctypes.c_int
            lib.oracle_loss_variant_paired.argtypes = [ctypes.c_int64, ctypes.c_int, P, P, P, P, ctypes.c_int, P, P,
                                                       P, P, P]
            lib.oracle_loss_variant_paired.restype = ctypes.c_int
            lib.oracle_loss_variant_pair_f64.argtypes = [ctypes.c_int, P, ctypes.c_int, P, ctypes.c_int,
                                                         ctypes.c_int, ctypes.c_double, P, P, P]
            lib.oracle_loss_variant_pair_f64.restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _u8(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.uint8)


def _chunks(n, threads):
    threads = max(1, min(threads, n)) if n > 0 else 1
    step = (n + threads - 1) // threads if n > 0 else 0
    return [(s, min(n, s + step)) for s in range(0, n, step)] if n > 0 else []


def iou_paired(p1, p2, c1=None, c2=None, threads: int = 1):
    """Forward on paired polygons [n, K, 2] (float32).

    Returns dict(iou=float64[n], nx=uint8[n], xflags=uint8[n, 2K],
    degen=uint8[n], areas=float64[n, 3] (A_i, A_1, A_2), status=int)."""
    lib = _load()
    p1, p2, c1, c2 = _f32(p1), _f32(p2), _u8(c1), _u8(c2)
    n, K = p1.shape[0], p1.shape[1]
    out = dict(iou=np.zeros(n, np.float64), nx=np.zeros(n, np.uint8),
               xflags=np.full((n, 2 * K), 0xFF, np.uint8), degen=np.zeros(n, np.uint8),
               areas=np.zeros((n, 3), np.float64))
    status = [0]

    def run(rng):
        s, e = rng
        m = e - s
        st = lib.oracle_iou_paired(
            m, K, _ptr(p1[s:e]), _ptr(None if c1 is None else c1[s:e]), _ptr(p2[s:e]),
            _ptr(None if c2 is None else c2[s:e]), _ptr(out["iou"][s:e]), _ptr(out["nx"][s:e]),
            _ptr(out["xflags"][s:e]), _ptr(out["degen"][s:e]), _ptr(out["areas"][s:e]))
        status[0] |= st

    _run_parallel(run, _chunks(n, threads))
    out["status"] = status[0]
    return out


def intersect_paired(p1, p2, c1=None, c2=None, threads: int = 1):
    """The intersection polygon of each pair (paper Sec. II-B `intersect`).

    Returns dict(verts=float64[n, 2K, 2] in xflags order, unused slots 0,
    nx=uint8[n], xflags=uint8[n, 2K], status=int)."""
    lib = _load()
    p1, p2, c1, c2 = _f32(p1), _f32(p2), _u8(c1), _u8(c2)
    n, K = p1.shape[0], p1.shape[1]
    out = dict(verts=np.zeros((n, 2 * K, 2), np.float64), nx=np.zeros(n, np.uint8),
               xflags=np.full((n, 2 * K), 0xFF, np.uint8))
    status = [0]

    def run(rng):
        s, e = rng
        st = lib.oracle_intersect_paired(
            e - s, K, _ptr(p1[s:e]), _ptr(None if c1 is None else c1[s:e]), _ptr(p2[s:e]),
            _ptr(None if c2 is None else c2[s:e]), _ptr(out["verts"][s:e]), _ptr(out["nx"][s:e]),
            _ptr(out["xflags"][s:e]))
        status[0] |= st

    _run_parallel(run, _chunks(n, threads))
    out["status"] = status[0]
    return out


def area(p, c=None):
    """Shoelace area of each polygon [n, K, 2] (paper Sec. II-B `area`)."""
    lib = _load()
    p, c = _f32(p), _u8(c)
    n, K = p.shape[0], p.shape[1]
    out = np.zeros(n, np.float64)
    lib.oracle_area(n, K, _ptr(p), _ptr(c), _ptr(out))
    return out


# ------------------------------------------------------------------ lines
#
# Lines (paper Sec. III, "Lines"): stored as the coefficients (a, b, c) of
# a x + b y + c = 0 and defined from two points differentiably.  Plain
# numpy in FP64; the gradients are the hand-derived adjoints of these
# formulas.

def line_from_points(p, q):
    """Line through p and q ([n, 2] each): (a, b, c) = (p_y - q_y, q_x - p_x,
    p_x q_y - q_x p_y), so that a x + b y + c = 0 on both points."""
    p = np.asarray(p, np.float64)
    q = np.asarray(q, np.float64)
    return np.stack([p[:, 1] - q[:, 1], q[:, 0] - p[:, 0], p[:, 0] * q[:, 1] - q[:, 0] * p[:, 1]], 1)


def line_from_points_backward(p, q, g):
    """dL/dp, dL/dq from dL/d(a, b, c) = g [n, 3]."""
    p = np.asarray(p, np.float64)
    q = np.asarray(q, np.float64)
    g = np.asarray(g, np.float64)
    ga, gb, gc = g[:, 0], g[:, 1], g[:, 2]
    gp = np.stack([-gb + gc * q[:, 1], ga - gc * q[:, 0]], 1)
    gq = np.stack([gb - gc * p[:, 1], -ga + gc * p[:, 0]], 1)
    return gp, gq


def line_intersect(l1, l2):
    """Intersection point of two lines ([n, 3] each): (X / W, Y / W) with
    X = b1 c2 - b2 c1, Y = c1 a2 - c2 a1, W = a1 b2 - a2 b1 (W = 0: parallel,
    non-finite result)."""
    l1 = np.asarray(l1, np.float64)
    l2 = np.asarray(l2, np.float64)
    a1, b1, c1 = l1[:, 0], l1[:, 1], l1[:, 2]
    a2, b2, c2 = l2[:, 0], l2[:, 1], l2[:, 2]
    W = a1 * b2 - a2 * b1
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.stack([(b1 * c2 - b2 * c1) / W, (c1 * a2 - c2 * a1) / W], 1)


def line_intersect_backward(l1, l2, g):
    """dL/dl1, dL/dl2 from dL/d(x, y) = g [n, 2]."""
    l1 = np.asarray(l1, np.float64)
    l2 = np.asarray(l2, np.float64)
    g = np.asarray(g, np.float64)
    a1, b1, c1 = l1[:, 0], l1[:, 1], l1[:, 2]
    a2, b2, c2 = l2[:, 0], l2[:, 1], l2[:, 2]
    W = a1 * b2 - a2 * b1
    x = (b1 * c2 - b2 * c1) / W
    y = (c1 * a2 - c2 * a1) / W
    gX, gY = g[:, 0] / W, g[:, 1] / W
    gW = -(g[:, 0] * x + g[:, 1] * y) / W
    gl1 = np.stack([-gY * c2 + gW * b2, gX * c2 - gW * a2, -gX * b2 + gY * a2], 1)
    gl2 = np.stack([gY * c1 - gW * b1, -gX * c1 + gW * a1, gX * b1 - gY * a1], 1)
    return gl1, gl2


def iou_backward_paired(p1, p2, grad, nx, xflags, c1=None, c2=None, threads: int = 1):
    """Backward on paired polygons; returns (g1, g2) float64 [n, K, 2]."""
    lib = _load()
    p1, p2, c1, c2 = _f32(p1), _f32(p2), _u8(c1), _u8(c2)
    grad = np.ascontiguousarray(grad, dtype=np.float64)
    nx = np.ascontiguousarray(nx, dtype=np.uint8)
    xflags = np.ascontiguousarray(xflags, dtype=np.uint8)
    n, K = p1.shape[0], p1.shape[1]
    g1 = np.zeros((n, K, 2), np.float64)
    g2 = np.zeros((n, K, 2), np.float64)

    def run(rng):
        s, e = rng
        lib.oracle_iou_backward_paired(
            e - s, K, _ptr(p1[s:e]), _ptr(None if c1 is None else c1[s:e]), _ptr(p2[s:e]),
            _ptr(None if c2 is None else c2[s:e]), _ptr(grad[s:e]), _ptr(nx[s:e]), _ptr(xflags[s:e]),
            _ptr(g1[s:e]), _ptr(g2[s:e]))

    _run_parallel(run, _chunks(n, threads))
    return g1, g2


def iou_pairwise(a, b, ca=None, cb=None, threads: int = 1):
    """N x M IoU matrix (float64) and nx (uint8)."""
    lib = _load()
    a, b, ca, cb = _f32(a), _f32(b), _u8(ca), _u8(cb)
    N, M, K = a.shape[0], b.shape[0], a.shape[1]
    iou = np.zeros((N, M), np.float64)
    nx = np.zeros((N, M), np.uint8)

    def run(rng):
        s, e = rng
        lib.oracle_iou_pairwise(e - s, M, K, _ptr(a[s:e]), _ptr(None if ca is None else ca[s:e]), _ptr(b),
                                _ptr(cb), _ptr(iou[s:e]), _ptr(nx[s:e]))

    _run_parallel(run, _chunks(N, threads))
    return iou, nx


def iou_pair_f64(p1, p2, K=None):
    """Single pair in double: returns (iou, ai, a1, a2, nx, codes, degen, status)."""
    lib = _load()
    p1 = np.ascontiguousarray(p1, dtype=np.float64)
    p2 = np.ascontiguousarray(p2, dtype=np.float64)
    n1, n2 = p1.shape[0], p2.shape[0]
    K = K or max(n1, n2)
    out = np.zeros(4, np.float64)
    nx = ctypes.c_int(0)
    dg = ctypes.c_int(0)
    code = np.full(2 * K, 0xFF, np.uint8)
    st = lib.oracle_iou_pair_f64(K, _ptr(p1), n1, _ptr(p2), n2, _ptr(out), ctypes.byref(nx), _ptr(code),
                                 ctypes.byref(dg))
    return out[0], out[1], out[2], out[3], nx.value, code, dg.value, st


def iou_backward_pair_f64(p1, p2, grad, nx, code, K=None):
    """Single pair backward in double; returns (g1 [n1,2], g2 [n2,2])."""
    lib = _load()
    p1 = np.ascontiguousarray(p1, dtype=np.float64)
    p2 = np.ascontiguousarray(p2, dtype=np.float64)
    n1, n2 = p1.shape[0], p2.shape[0]
    K = K or max(n1, n2)
    code = np.ascontiguousarray(code, dtype=np.uint8)
    g1 = np.zeros((K, 2), np.float64)
    g2 = np.zeros((K, 2), np.float64)
    lib.oracle_iou_backward_pair_f64(K, _ptr(p1), n1, _ptr(p2), n2, float(grad), int(nx), _ptr(code), _ptr(g1),
                                     _ptr(g2))
    return g1[:n1], g2[:n2]


def _run_parallel(fn, ranges):
    if len(ranges) <= 1:
        for r in ranges:
            fn(r)
        return
    # ctypes releases the GIL during the foreign call, so threads use all cores.
    with ThreadPoolExecutor(max_workers=len(ranges)) as ex:
        list(ex.map(fn, ranges))


def iou_loss(p1, p2, weight=None, scale=1.0, c1=None, c2=None, threads: int = 1):
    """IoU loss of the paper's case study (Sec. IV-A) in FP64:
    loss = scale * sum_k w_k (1 - IoU_k), and its gradient, i.e. the pinned
    backward with dL/dIoU_k = -scale w_k.  Returns (loss, g1, g2, forward dict)."""
    n = np.asarray(p1).shape[0]
    w = np.ones(n) if weight is None else np.asarray(weight, dtype=np.float64)
    f = iou_paired(p1, p2, c1, c2, threads=threads)
    loss = float(scale * np.sum(w * (1.0 - f["iou"])))
    g1, g2 = iou_backward_paired(p1, p2, -scale * w, f["nx"], f["xflags"], c1, c2, threads=threads)
    return loss, g1, g2, f


def area_backward_paired(p1, p2, gai, ga1, ga2, nx, xflags, c1=None, c2=None, threads: int = 1):
    """Area adjoint on paired polygons: dL/dA_i, dL/dA_1, dL/dA_2 [n] -> (g1, g2)
    float64 [n, K, 2] through the recorded (nx, xflags)."""
    lib = _load()
    p1, p2, c1, c2 = _f32(p1), _f32(p2), _u8(c1), _u8(c2)
    gai, ga1, ga2 = (np.ascontiguousarray(g, dtype=np.float64) for g in (gai, ga1, ga2))
    nx = np.ascontiguousarray(nx, dtype=np.uint8)
    xflags = np.ascontiguousarray(xflags, dtype=np.uint8)
    n, K = p1.shape[0], p1.shape[1]
    g1 = np.zeros((n, K, 2), np.float64)
    g2 = np.zeros((n, K, 2), np.float64)

    def run(rng):
        s, e = rng
        lib.oracle_area_backward_paired(
            e - s, K, _ptr(p1[s:e]), _ptr(None if c1 is None else c1[s:e]), _ptr(p2[s:e]),
            _ptr(None if c2 is None else c2[s:e]), _ptr(gai[s:e]), _ptr(ga1[s:e]), _ptr(ga2[s:e]), _ptr(nx[s:e]),
            _ptr(xflags[s:e]), _ptr(g1[s:e]), _ptr(g2[s:e]))

    _run_parallel(run, _chunks(n, threads))
    return g1, g2


# ----------------------------------------------------------------- 3D IoU
#
# 3D IoU of boxes given as a bird's-eye-view polygon and a vertical extent
# (z_center, height) (the rotated 3D IoU loss of the paper's Sec. IV-A): the
# intersection volume is A_i * ov with ov the overlap of the two z-intervals,
# IoU3 = A_i ov / (A_1 h_1 + A_2 h_2 - A_i ov), 0 when that union is not
# positive.  At equal interval ends the subgradient takes P1's end.

def _z_terms(z1, z2):
    z1 = np.asarray(z1, dtype=np.float64)
    z2 = np.asarray(z2, dtype=np.float64)
    lo1, hi1 = z1[:, 0] - 0.5 * z1[:, 1], z1[:, 0] + 0.5 * z1[:, 1]
    lo2, hi2 = z2[:, 0] - 0.5 * z2[:, 1], z2[:, 0] + 0.5 * z2[:, 1]
    top1 = hi1 <= hi2  # P1's top is the overlap's top
    bot1 = lo1 >= lo2  # P1's bottom is the overlap's bottom
    ov = np.minimum(hi1, hi2) - np.maximum(lo1, lo2)
    return z1[:, 1], z2[:, 1], np.maximum(ov, 0.0), ov > 0.0, top1, bot1


def iou3d_paired(p1, p2, z1, z2, c1=None, c2=None, threads: int = 1):
    """3D IoU of paired boxes; returns the 2D forward's dict with iou replaced
    by the 3D IoU and the vertical overlap added as "ov"."""
    f = iou_paired(p1, p2, c1, c2, threads=threads)
    h1, h2, ov, _, _, _ = _z_terms(z1, z2)
    ai, a1, a2 = f["areas"][:, 0], f["areas"][:, 1], f["areas"][:, 2]
    inter = np.where(f["nx"] >= 3, ai, 0.0) * ov
    union = a1 * h1 + a2 * h2 - inter
    with np.errstate(divide="ignore", invalid="ignore"):
        f["iou"] = np.where(union > 0.0, inter / union, 0.0)
    f["ov"] = ov
    return f


def iou3d_backward_paired(p1, p2, z1, z2, grad, nx, xflags, c1=None, c2=None, threads: int = 1):
    """dL/dIoU3 [n] -> (g1 [n,K,2], gz1 [n,2], g2 [n,K,2], gz2 [n,2]) in float64,
    gz = dL/d(z_center, height)."""
    f = iou_paired(p1, p2, c1, c2, threads=threads)
    g = np.asarray(grad, dtype=np.float64)
    h1, h2, ov, pos, top1, bot1 = _z_terms(z1, z2)
    ai = np.where(np.asarray(nx) >= 3, f["areas"][:, 0], 0.0)
    a1, a2 = f["areas"][:, 1], f["areas"][:, 2]
    inter = ai * ov
    v1, v2 = a1 * h1, a2 * h2
    union = v1 + v2 - inter
    ok = union > 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        d_inter = np.where(ok, (v1 + v2) / union ** 2, 0.0)  # dIoU3 / d(A_i ov)
        d_vol = np.where(ok, -inter / union ** 2, 0.0)  # dIoU3 / dV_k
    gai = g * d_inter * ov
    ga1 = g * d_vol * h1
    ga2 = g * d_vol * h2
    g1, g2 = area_backward_paired(p1, p2, gai, ga1, ga2, nx, xflags, c1, c2, threads=threads)
    # ov = min(hi1, hi2) - max(lo1, lo2), hi = z + h/2, lo = z - h/2
    gov = np.where(pos, g * d_inter * ai, 0.0)
    t1, b1 = top1.astype(np.float64), bot1.astype(np.float64)
    gz1 = np.stack([gov * (t1 - b1), gov * 0.5 * (t1 + b1) + g * d_vol * a1], axis=1)
    gz2 = np.stack([gov * ((1 - t1) - (1 - b1)), gov * 0.5 * ((1 - t1) + (1 - b1)) + g * d_vol * a2], axis=1)
    return g1, gz1, g2, gz2


# ------------------------------------------------------------ rotated NMS
#
# Greedy non-maximum suppression over rotated boxes (the consumer of the
# pairwise IoU matrix named in the paper's Sec. IV, OpenPCDet's rotated NMS):
# visit the boxes by descending score (equal scores: lower index first); keep
# a box unless a kept box overlaps it with IoU > threshold.

def nms_rotated(boxes, scores, threshold, counts=None, threads: int = 1):
    """Kept box indices (int64, in visiting order)."""
    boxes = np.asarray(boxes)
    scores = np.asarray(scores, dtype=np.float64)
    n = boxes.shape[0]
    if n == 0:
        return np.zeros(0, np.int64)
    order = np.array(sorted(range(n), key=lambda i: (-scores[i], i)), dtype=np.int64)
    cs = None if counts is None else np.asarray(counts)[order]
    iou, _ = iou_pairwise(boxes[order], boxes[order], cs, cs, threads=threads)
    removed = np.zeros(n, bool)
    keep = []
    for a in range(n):
        if removed[a]:
            continue
        keep.append(order[a])
        removed[a + 1:] |= iou[a, a + 1:] > threshold
    return np.array(keep, dtype=np.int64)


GIOU = 1
DIOU = 2


def loss_variant_paired(p1, p2, variant, weight=None, c1=None, c2=None, threads: int = 1):
    """Per-pair loss terms of the GIoU (variant 1) or DIoU (variant 2) loss and
    their gradients (dgal_oracle.c, "GIoU / DIoU terms of the loss").

    Returns dict(lk=float64[n] = w (1 - GIoU) or w (1 - DIoU),
    terms=float64[n, 4] = (IoU, hull area, rho2, c2), g1, g2 = float64[n, K, 2]
    = d lk / d p1, d p2, status=int)."""
    lib = _load()
    p1, p2, c1, c2 = _f32(p1), _f32(p2), _u8(c1), _u8(c2)
    n, K = p1.shape[0], p1.shape[1]
    w = None if weight is None else np.ascontiguousarray(weight, dtype=np.float64)
    out = dict(lk=np.zeros(n), terms=np.zeros((n, 4)), g1=np.zeros((n, K, 2)), g2=np.zeros((n, K, 2)))
    status = [0]

    def run(rng):
        s, e = rng
        st = lib.oracle_loss_variant_paired(
            e - s, K, _ptr(p1[s:e]), _ptr(None if c1 is None else c1[s:e]), _ptr(p2[s:e]),
            _ptr(None if c2 is None else c2[s:e]), int(variant), _ptr(None if w is None else w[s:e]),
            _ptr(out["lk"][s:e]), _ptr(out["terms"][s:e]), _ptr(out["g1"][s:e]), _ptr(out["g2"][s:e]))
        status[0] |= st

    _run_parallel(run, _chunks(n, threads))
    out["status"] = status[0]
    return out


def loss_variant_pair_f64(p1, p2, variant, w=1.0, K=None):
    """Single pair in double: returns (lk, g1 [n1, 2], g2 [n2, 2])."""
    lib = _load()
    p1 = np.ascontiguousarray(p1, dtype=np.float64)
    p2 = np.ascontiguousarray(p2, dtype=np.float64)
    n1, n2 = p1.shape[0], p2.shape[0]
    K = K or max(n1, n2)
    lk = ctypes.c_double(0.0)
    g1 = np.zeros((K, 2), np.float64)
    g2 = np.zeros((K, 2), np.float64)
    lib.oracle_loss_variant_pair_f64(K, _ptr(p1), n1, _ptr(p2), n2, int(variant), float(w), ctypes.byref(lk),
                                     _ptr(g1), _ptr(g2))
    return lk.value, g1[:n1], g2[:n2]
