"""GPU parity of the IoU loss call (loss-mode forward, loss-mode backward,
deterministic partial sum)."""
import numpy as np
import pytest

from paper_2011_11134_gb300 import workloads as W

from .gpu_helpers import GRAD_RTOL, IOU_ATOL, THREADS, dev, grad_rel_err, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_11134_gb300 as m

    m.dgal_get_device_status(clear=True)
    return m


@pytest.mark.parametrize("n", [200_000, 4096 + 37])
def test_fused_loss_matches_oracle_and_unfused(dg, orc, n):
    import torch

    d = W.loss_pairs_1m(seed=3, n=n)
    w = np.linspace(0.2, 1.8, n).astype(np.float32)
    scale = 1.0 / n
    p1, p2, wt = dev(d["p1"]), dev(d["p2"]), dev(w)
    loss, g1, g2, iou = dg.dgal_iou_loss(p1, p2, wt, scale, with_iou=True)
    ref_loss, r1, r2, f = orc.iou_loss(d["p1"], d["p2"], weight=w.astype(np.float64), scale=scale, threads=THREADS)
    # each IoU is within IOU_ATOL, so the weighted mean is within IOU_ATOL * mean|w|
    assert abs(host(loss)[0] - ref_loss) <= IOU_ATOL * scale * np.abs(w).sum() + 1e-6 * abs(ref_loss)
    assert np.abs(host(iou) - f["iou"]).max() <= IOU_ATOL
    gen = f["degen"] == 0
    rel = grad_rel_err(host(g1), host(g2), r1, r2, gen)
    assert rel.max() <= GRAD_RTOL, rel.max()
    # same gradients as the separate forward + backward with dL/dIoU = -scale w
    iv, nx, xf, _ = dg.dgal_iou_paired(p1, p2)
    b1, b2 = dg.dgal_iou_backward(p1, p2, -scale * wt, nx, xf)
    assert torch.equal(iv, iou)
    m = max(b1.abs().max().item(), b2.abs().max().item())
    assert (b1 - g1).abs().max().item() <= 1e-6 * m and (b2 - g2).abs().max().item() <= 1e-6 * m
    # deterministic reduction
    loss2, _, _, _ = dg.dgal_iou_loss(p1, p2, wt, scale)
    assert torch.equal(loss, loss2)


def test_fused_loss_autograd_and_edges(dg):
    import torch

    d = W.paired_rect_4096(seed=4, n=999)
    p1 = dev(d["p1"]).requires_grad_(True)
    p2 = dev(d["p2"]).requires_grad_(True)
    loss = dg.iou_loss(p1, p2, reduction="mean")
    (3.0 * loss).backward()
    _, g1, g2, _ = dg.dgal_iou_loss(p1.detach(), p2.detach(), None, 1.0 / 999)
    assert torch.allclose(p1.grad, 3.0 * g1, rtol=1e-6, atol=0) and torch.allclose(p2.grad, 3.0 * g2, rtol=1e-6, atol=0)
    z = torch.zeros((0, 4, 2), device="cuda")
    lz, _, _, _ = dg.dgal_iou_loss(z, z)
    assert host(lz)[0] == 0.0
    with pytest.raises(dg.DgalError):
        dg.dgal_iou_loss(p1.detach(), p2.detach(), workspace=torch.empty(16, device="cuda", dtype=torch.uint8))


def test_loss_k8_counts_matches_oracle(dg, orc):
    import torch

    d = W.convex_pairs_4m(seed=5, n=60_000)
    n = d["p1"].shape[0]
    w = np.linspace(0.5, 1.5, n).astype(np.float32)
    p1, p2, c1, c2 = dev(d["p1"]), dev(d["p2"]), dev(d["c1"]), dev(d["c2"])
    loss, g1, g2, iou = dg.dgal_iou_loss(p1, p2, dev(w), 2.0, c1=c1, c2=c2, with_iou=True)
    ref_loss, r1, r2, f = orc.iou_loss(d["p1"], d["p2"], weight=w.astype(np.float64), scale=2.0, c1=d["c1"],
                                       c2=d["c2"], threads=THREADS)
    assert abs(host(loss)[0] - ref_loss) <= IOU_ATOL * 2.0 * np.abs(w).sum() + 1e-6 * abs(ref_loss)
    assert np.abs(host(iou) - f["iou"]).max() <= IOU_ATOL
    _, nx, xf, degen = dg.dgal_iou_paired(p1, p2, c1, c2, with_degen=True)
    gen = (f["degen"] == 0) & (host(degen) == 0)
    rel = grad_rel_err(host(g1), host(g2), r1, r2, gen)
    assert rel.max() <= GRAD_RTOL, rel.max()
    b1, b2 = dg.dgal_iou_backward(p1, p2, -2.0 * dev(w), nx, xf, c1=c1, c2=c2)
    assert torch.equal(b1, g1) and torch.equal(b2, g2)
