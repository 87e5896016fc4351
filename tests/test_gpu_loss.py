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
    # the loss takes one thread per pair at every size; below the paired
    # calls' group threshold those take a group of 8 lanes per pair, whose
    # FP32 sums round in another order
    if n >= dg.dgal_get_paired_config(4)["group_below"]:
        assert torch.equal(iv, iou)
    else:
        assert (iv - iou).abs().max().item() <= 1e-6
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
    # the upstream factor enters dL/dIoU inside the library: equal up to rounding
    tol = 1e-6 * 3.0 * max(g1.abs().max().item(), g2.abs().max().item())
    assert (p1.grad - 3.0 * g1).abs().max().item() <= tol and (p2.grad - 3.0 * g2).abs().max().item() <= tol
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
    # the same gradients up to rounding (the loss-mode kernels are compiled
    # with the GIoU term of the adjoint, which can move a contraction)
    m = max(b1.abs().max().item(), b2.abs().max().item())
    assert (b1 - g1).abs().max().item() <= 1e-6 * m and (b2 - g2).abs().max().item() <= 1e-6 * m


@pytest.mark.parametrize("variant", ["giou", "diou"])
@pytest.mark.parametrize("K", [4, 8])
def test_loss_variants_match_oracle(dg, orc, variant, K):
    """GIoU / DIoU loss: the loss value and the gradients against the oracle's
    per-pair terms (gradients on pairs the oracle does not flag; for DIoU also
    leaving out pairs whose diameter is a near-tie, where it has no
    derivative)."""
    import torch

    if K == 4:
        d = W.loss_pairs_1m(seed=21, n=50_000)
        c1 = c2 = None
    else:
        d = W.convex_pairs_4m(seed=21, n=30_000)
        c1, c2 = d["c1"], d["c2"]
    n = d["p1"].shape[0]
    w = np.linspace(0.5, 1.5, n).astype(np.float32)
    scale = 1.0 / n
    v = 1 if variant == "giou" else 2
    p1, p2, wt = dev(d["p1"]), dev(d["p2"]), dev(w)
    dc1 = None if c1 is None else dev(c1)
    dc2 = None if c2 is None else dev(c2)
    loss, g1, g2, _ = dg.dgal_iou_loss(p1, p2, wt, scale, dc1, dc2, variant=variant)
    ref = orc.loss_variant_paired(d["p1"], d["p2"], v, weight=w.astype(np.float64), c1=c1, c2=c2, threads=THREADS)
    ref_loss = scale * ref["lk"].sum()
    # each term is within a few IOU_ATOL of the oracle's
    assert abs(host(loss)[0] - ref_loss) <= 4 * IOU_ATOL * scale * np.abs(w).sum() + 1e-6 * abs(ref_loss)
    f = orc.iou_paired(d["p1"], d["p2"], c1, c2, threads=THREADS)
    keep = f["degen"] == 0
    if v == 2:
        pts = np.concatenate([d["p1"], d["p2"]], 1).astype(np.float64)
        if c1 is not None:
            K_ = d["p1"].shape[1]
            live = np.concatenate([np.arange(K_)[None] < c1[:, None], np.arange(K_)[None] < c2[:, None]], 1)
        else:
            live = np.ones(pts.shape[:2], bool)
        dd = ((pts[:, :, None, :] - pts[:, None, :, :]) ** 2).sum(-1)
        m = pts.shape[1]
        iu = np.triu_indices(m, 1)
        pair_live = live[:, iu[0]] & live[:, iu[1]]
        vals = np.where(pair_live, dd[:, iu[0], iu[1]], -1.0)
        top = np.sort(vals, axis=1)
        keep &= top[:, -1] - top[:, -2] >= 1e-4 * top[:, -1]
    assert keep.mean() > 0.5
    rel = grad_rel_err(host(g1), host(g2), scale * ref["g1"], scale * ref["g2"], keep)
    assert rel.max() <= GRAD_RTOL, f"{variant} K={K}: max grad rel err {rel.max():.3e}"
    # deterministic
    loss2, _, _, _ = dg.dgal_iou_loss(p1, p2, wt, scale, dc1, dc2, variant=variant)
    assert torch.equal(loss, loss2)
    assert dg.dgal_get_device_status() == 0


@pytest.mark.parametrize("variant", ["iou", "giou", "diou"])
def test_loss_backward_takes_upstream_gradient_on_device(dg, variant):
    """The autograd loss runs the forward alone and, in the backward,
    dgal_iou_loss_backward with the incoming gradient read on the device: its
    gradients equal the one-call gradients times that gradient."""
    import torch

    d = W.paired_rect_4096(seed=8, n=3001)
    p1 = dev(d["p1"]).requires_grad_(True)
    p2 = dev(d["p2"]).requires_grad_(True)
    loss = dg.iou_loss(p1, p2, reduction="mean", variant=variant)
    (2.5 * loss).backward()
    l0, g1, g2, _ = dg.dgal_iou_loss(p1.detach(), p2.detach(), None, 1.0 / 3001, variant=variant)
    assert torch.equal(loss.detach().reshape(1), l0)
    tol = 1e-6 * 2.5 * max(g1.abs().max().item(), g2.abs().max().item())
    assert (p1.grad - 2.5 * g1).abs().max().item() <= tol and (p2.grad - 2.5 * g2).abs().max().item() <= tol
    # the two variant flags exclude each other
    L = dg._lib
    ws = torch.empty(dg.dgal_iou_loss_workspace_bytes(3001, 4), device="cuda", dtype=torch.uint8)
    with pytest.raises(dg.DgalError):
        L.call("dgal_iou_loss", L.ptr(p1.detach()), None, L.ptr(p2.detach()), None, 3001, 4, None, 1.0,
               L.ptr(torch.empty(1, device="cuda")), None, None, None, L.ptr(ws), ws.numel(),
               dg.DGAL_LOSS_GIOU | dg.DGAL_LOSS_DIOU, L.stream_ptr())


def test_giou_diou_special_cases(dg):
    """Identical boxes: 0 for both losses; disjoint boxes: GIoU loss 1 + (A_h -
    U) / A_h > 1 and DIoU loss 1 + rho2 / c2; the 3D loss refuses the
    variants."""
    import torch

    P = torch.tensor([[[0, 0], [2, 0], [2, 2], [0, 2]]], dtype=torch.float32, device="cuda")
    Q = P + torch.tensor([3.0, 0.0], device="cuda")
    for v in ("giou", "diou"):
        l, _, _, _ = dg.dgal_iou_loss(P, P.clone(), variant=v)
        assert abs(l.item()) <= 1e-6
    l, _, _, _ = dg.dgal_iou_loss(P, Q, variant="giou")
    # hull of [0,2]^2 and [3,5]x[0,2] is [0,5]x[0,2]: A_h = 10, U = 8
    assert l.item() == pytest.approx(1.0 + 2.0 / 10.0, abs=1e-6)
    l, _, _, _ = dg.dgal_iou_loss(P, Q, variant="diou")
    # centres 3 apart, diameter from (0,0) to (5,2): c2 = 29
    assert l.item() == pytest.approx(1.0 + 9.0 / 29.0, abs=1e-6)
    z = torch.zeros((1, 2), device="cuda")
    with pytest.raises(dg.DgalError):
        dg._lib.call("dgal_iou3d_loss", dg._lib.ptr(P), None, dg._lib.ptr(z), dg._lib.ptr(Q), None, dg._lib.ptr(z), 1,
                     4, None, 1.0, dg._lib.ptr(torch.empty(1, device="cuda")), None, None, None, None, None,
                     dg._lib.ptr(torch.empty(1 << 16, device="cuda", dtype=torch.uint8)), 1 << 16,
                     dg.DGAL_LOSS_GIOU, dg._lib.stream_ptr())
