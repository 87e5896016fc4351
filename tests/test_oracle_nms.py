"""Pins for the oracle's rotated NMS: an independent closed-form IoU on
axis-aligned boxes, the greedy invariants, and the threshold extremes."""
import numpy as np

from paper_2011_11134_gb300 import workloads as W


def _greedy(iou_sorted, order, thr):
    n = len(order)
    keep, removed = [], np.zeros(n, bool)
    for a in range(n):
        if not removed[a]:
            keep.append(order[a])
            for b in range(a + 1, n):
                if iou_sorted[a, b] > thr:
                    removed[b] = True
    return keep


def test_axis_aligned_closed_form(orc):
    r = np.random.default_rng(41)
    n = 300
    c = r.uniform(0, 20, (n, 2))
    wh = r.uniform(0.5, 4.0, (n, 2))
    lo, hi = (c - wh / 2).astype(np.float32), (c + wh / 2).astype(np.float32)
    boxes = np.stack([lo, np.stack([hi[:, 0], lo[:, 1]], 1), hi, np.stack([lo[:, 0], hi[:, 1]], 1)], 1)
    scores = r.permutation(n).astype(np.float32)  # distinct scores
    order = np.argsort(-scores, kind="stable")
    L, H = lo.astype(np.float64)[order], hi.astype(np.float64)[order]
    ext = np.clip(np.minimum(H[:, None], H[None]) - np.maximum(L[:, None], L[None]), 0, None)
    inter = ext[..., 0] * ext[..., 1]
    area = (H - L).prod(1)
    iou = inter / (area[:, None] + area[None] - inter)
    for thr in (0.1, 0.3, 0.5):
        ref = _greedy(iou, order, thr)
        got = orc.nms_rotated(boxes, scores, thr)
        assert list(got) == list(ref)


def test_invariants_and_extremes(orc):
    d = W.pairwise_bev_2000(seed=42)
    boxes = d["a"][:600]
    r = np.random.default_rng(43)
    scores = r.uniform(0, 1, 600).astype(np.float32)
    scores[::7] = scores[0]  # ties: lower index first
    thr = 0.2
    keep = orc.nms_rotated(boxes, scores, thr)
    iou, _ = orc.iou_pairwise(boxes, boxes)
    # kept boxes do not overlap each other above the threshold
    kk = iou[np.ix_(keep, keep)]
    assert (kk[~np.eye(len(keep), dtype=bool)] <= thr).all()
    # every dropped box overlaps an earlier-visited kept box above the threshold
    rank = {int(i): (-float(scores[i]), int(i)) for i in range(600)}
    kept = set(int(k) for k in keep)
    for i in range(600):
        if i in kept:
            continue
        assert any(iou[k, i] > thr and rank[k] < rank[i] for k in kept)
    # kept order is the visiting order
    assert [rank[int(k)] for k in keep] == sorted(rank[int(k)] for k in keep)
    assert len(orc.nms_rotated(boxes, scores, 1.0)) == 600  # IoU never exceeds 1
    top = orc.nms_rotated(boxes, scores, -0.5)  # every pair "overlaps": only the first visited box stays
    assert list(top) == [min(range(600), key=lambda i: rank[i])]
