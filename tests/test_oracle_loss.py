"""Pins for the oracle's IoU-loss composition: loss values on constructed
cases, and the loss gradient against central differences of the loss."""
import numpy as np

from paper_2011_11134_gb300 import workloads as W


def test_loss_special_cases(orc):
    d = W.paired_rect_4096(seed=21, n=200)
    loss, g1, g2, _ = orc.iou_loss(d["p1"], d["p1"])  # identical pairs: IoU = 1
    assert abs(loss) <= 1e-10
    far = d["p2"] + np.float32(100.0)
    w = np.linspace(0.5, 2.0, 200)
    loss, g1, g2, _ = orc.iou_loss(d["p1"], far, weight=w, scale=0.25)  # disjoint: IoU = 0
    assert abs(loss - 0.25 * w.sum()) <= 1e-10
    assert np.abs(g1).max() == 0 and np.abs(g2).max() == 0


def test_loss_gradient_finite_differences(orc):
    d = W.loss_pairs_1m(seed=22, n=40)
    w = np.linspace(0.3, 1.7, 40)
    loss, g1, g2, f = orc.iou_loss(d["p1"], d["p2"], weight=w, scale=0.5)
    checked = 0
    for k in range(40):
        if f["degen"][k] or f["nx"][k] == 0:
            continue
        P, Q = d["p1"][k].astype(np.float64), d["p2"][k].astype(np.float64)
        h = 1e-6 * max(np.abs(P - P[0]).max(), np.abs(Q - P[0]).max())
        num = np.zeros((2, 4, 2))
        ok = True
        for which in range(2):
            for v in range(4):
                for c in range(2):
                    vals = []
                    for sg in (1, -1):
                        A, B = P.copy(), Q.copy()
                        (A if which == 0 else B)[v, c] += sg * h
                        r = orc.iou_pair_f64(A, B, 4)
                        ok &= r[4] == f["nx"][k] and list(r[5]) == list(f["xflags"][k])
                        vals.append(0.5 * w[k] * (1.0 - r[0]))
                    num[which, v, c] = (vals[0] - vals[1]) / (2 * h)
        if not ok:
            continue
        G = np.stack([g1[k], g2[k]])
        assert np.abs(G - num).max() <= 1e-6 * max(np.abs(num).max(), 1e-9)
        checked += 1
    assert checked >= 30
