"""GPU parity of the rotated NMS (dgal_nms_rotated) against the oracle's
greedy NMS on the FP64 IoU, and against the same greedy rule applied to the
library's own FP32 pairwise matrix.

The keep decision compares an IoU with the threshold.  The GPU decides on its
FP32 IoU (within 1e-5 of the FP64 value), the oracle on the FP64 IoU; the two
lists must be identical whenever no pair's FP64 IoU lies within that
tolerance of the threshold, which every case below checks first."""
import numpy as np
import pytest

from paper_2011_11134_gb300 import workloads as W

from .gpu_helpers import IOU_ATOL, THREADS, dev, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_11134_gb300 as m

    m.dgal_get_device_status(clear=True)
    return m


def _visit_order(scores):
    key = np.where(np.isnan(scores), -np.inf, scores.astype(np.float64))
    return np.array(sorted(range(len(scores)), key=lambda i: (-key[i], i)), dtype=np.int64)


def _greedy(iou, order, thr):
    """Greedy NMS on a full IoU matrix (indexed by box) in a given visiting order."""
    n = len(order)
    sub = iou[np.ix_(order, order)] > thr
    removed = np.zeros(n, bool)
    keep = []
    for a in range(n):
        if removed[a]:
            continue
        keep.append(int(order[a]))
        removed[a + 1:] |= sub[a, a + 1:]
    return keep


def _check(dg, orc, boxes, scores, thr, counts=None, label=""):
    import torch

    b, s = dev(boxes), dev(scores)
    c = dev(counts) if counts is not None else None
    keep = host(dg.dgal_nms_rotated(b, s, thr, counts=c)).tolist()
    # same rule on the library's own FP32 matrix: exact
    m, _ = dg.dgal_iou_pairwise(b, b, c, c, with_nx=False)
    torch.cuda.synchronize()
    order = _visit_order(scores)
    assert keep == _greedy(host(m), order, thr), f"{label}: differs from greedy on the FP32 pairwise matrix"
    # against the oracle: exact when no FP64 IoU is within the tolerance of thr
    ref_iou, _ = orc.iou_pairwise(boxes, boxes, counts, counts, threads=THREADS)
    band = np.abs(ref_iou - thr) <= IOU_ATOL
    np.fill_diagonal(band, False)
    assert not band.any(), f"{label}: a pair's IoU is within {IOU_ATOL} of the threshold; pick another seed"
    sc = np.where(np.isnan(scores), -np.inf, scores).astype(np.float32)
    ref = orc.nms_rotated(boxes, sc, thr, counts, threads=THREADS).tolist()
    assert keep == ref, f"{label}: {len(keep)} kept vs oracle {len(ref)}"
    return keep


@pytest.mark.parametrize("thr", [0.1, 0.2, 0.5, 0.8])
def test_nms_bev_2000(dg, orc, thr):
    d = W.pairwise_bev_2000(seed=7)
    boxes = d["a"]
    r = np.random.default_rng(70)
    scores = r.uniform(0, 1, len(boxes)).astype(np.float32)
    scores[::11] = scores[3]  # ties: lower index first
    keep = _check(dg, orc, boxes, scores, thr, label=f"bev thr={thr}")
    assert 0 < len(keep) < len(boxes)


def test_nms_k8_counts(dg, orc):
    d = W.convex_pairs_4m(seed=5, n=700, degenerate_frac=0.0)
    r = np.random.default_rng(71)
    scores = r.uniform(0, 1, 700).astype(np.float32)
    keep = _check(dg, orc, d["p1"], scores, 0.35, counts=d["c1"], label="K=8 counts")
    assert 0 < len(keep) < 700


def test_nms_wide_2600(dg, orc):
    """2600 boxes: 41 words per row, so the greedy pass also ORs words beyond
    the 32 it holds in registers for each 64-row block."""
    d = W.pairwise_bev_2000(seed=13, N=2600, M=1)
    r = np.random.default_rng(73)
    scores = r.uniform(0, 1, 2600).astype(np.float32)
    keep = _check(dg, orc, d["a"], scores, 0.3, label="2600 boxes")
    assert 0 < len(keep) < 2600


def test_nms_4500_far_words(dg, orc):
    """4500 boxes: 71 words per row, most of them beyond the 32 the greedy
    pass stages for each 64-row block."""
    d = W.pairwise_bev_2000(seed=20, N=4500, M=1)
    r = np.random.default_rng(74)
    scores = r.uniform(0, 1, 4500).astype(np.float32)
    scores[::7] = scores[5]  # ties: lower index first
    keep = _check(dg, orc, d["a"], scores, 0.45, label="4500 boxes")
    assert 0 < len(keep) < 4500


@pytest.mark.parametrize("n", [1, 2, 63, 64, 65, 129, 200])
def test_nms_ragged_sizes(dg, orc, n):
    d = W.pairwise_bev_2000(seed=100 + n, N=n, M=1)
    r = np.random.default_rng(n)
    scores = r.uniform(0, 1, n).astype(np.float32)
    # a small plane so that the boxes overlap
    boxes = (d["a"] - d["a"].reshape(-1, 2).min(0)) * np.float32(0.25)
    _check(dg, orc, boxes.astype(np.float32), scores, 0.1, label=f"n={n}")


def test_nms_nan_scores_and_extremes(dg, orc):
    import torch

    d = W.pairwise_bev_2000(seed=9, N=300, M=1)
    boxes = d["a"]
    r = np.random.default_rng(72)
    scores = r.uniform(0, 1, 300).astype(np.float32)
    scores[[5, 17, 250]] = np.nan  # visited last, as -infinity
    _check(dg, orc, boxes, scores, 0.2, label="NaN scores")
    b, s = dev(boxes), dev(scores)
    order = _visit_order(scores)
    assert host(dg.dgal_nms_rotated(b, s, 1.5)).tolist() == order.tolist()  # IoU never exceeds 1.5
    assert host(dg.dgal_nms_rotated(b, s, -0.5)).tolist() == [int(order[0])]  # every pair "overlaps"
    empty = torch.empty((0, 4, 2), device="cuda", dtype=torch.float32)
    assert dg.dgal_nms_rotated(empty, torch.empty(0, device="cuda"), 0.5).numel() == 0
    assert dg.dgal_get_device_status() == 0


def test_nms_wait_expiry_path(dg):
    """The greedy pass's bounded-wait failure path, reached without stalling
    anything: the test flag takes it at the second block once that block's
    copies have landed.  The call returns, the status word holds
    DGAL_DEV_TIMEOUT, the kept list stops after the first block (a prefix of
    the full result), and the next call on the same context gives the full
    result (the pass waited for its copies in flight before it stopped)."""
    import torch

    d = W.pairwise_bev_2000(seed=0)
    a = dev(d["a"])
    scores = torch.from_numpy(np.random.default_rng(0).uniform(0, 1, a.shape[0]).astype(np.float32)).cuda()
    full = dg.dgal_nms_rotated(a, scores, 0.2)
    dg.dgal_get_device_status(clear=True)
    keep, num = dg.dgal_nms_rotated(a, scores, 0.2, flags=dg.DGAL_FP64_REFINE | dg.DGAL_TEST_EXPIRE_WAIT,
                                    sync=False)
    torch.cuda.synchronize()
    assert dg.dgal_get_device_status(clear=True) & dg.DGAL_DEV_TIMEOUT
    m = int(num.item())
    assert 0 < m <= 64 and m < full.numel()
    assert torch.equal(keep[:m], full[:m])
    again = dg.dgal_nms_rotated(a, scores, 0.2)
    assert torch.equal(again, full)
    assert dg.dgal_get_device_status() == 0
