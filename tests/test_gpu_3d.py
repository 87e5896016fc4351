"""GPU parity of the 3D IoU (bird's-eye-view polygon x vertical extent), its
backward, and the 3D IoU loss, against the FP64 oracle."""
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


def _zrel(gz, rz, G, R, mask):
    """Per-pair relative error of all gradients (vertices and z) together."""
    A = np.concatenate([G.reshape(G.shape[0], -1), gz.reshape(gz.shape[0], -1)], 1).astype(np.float64)[mask]
    B = np.concatenate([R.reshape(R.shape[0], -1), rz.reshape(rz.shape[0], -1)], 1)[mask]
    return np.abs(A - B).max(1) / np.maximum(np.abs(B).max(1), 1e-6)


@pytest.mark.parametrize("n", [150_000, 4096 + 19])
def test_iou3d_forward_backward_k4(dg, orc, n):
    d = W.loss3d_pairs_1m(seed=8, n=n)
    p1, p2, z1, z2 = (dev(d[k]) for k in ("p1", "p2", "z1", "z2"))
    iou, nx, xf, degen = dg.dgal_iou3d_paired(p1, z1, p2, z2, with_degen=True)
    ref = orc.iou3d_paired(d["p1"], d["p2"], d["z1"], d["z2"], threads=THREADS)
    assert np.abs(host(iou) - ref["iou"]).max() <= IOU_ATOL
    gen = (ref["degen"] == 0) & (host(degen) == 0)
    assert (host(nx)[gen] == ref["nx"][gen]).all() and (host(xf)[gen] == ref["xflags"][gen]).all()
    # the bird's-eye-view state is the 2D forward's
    _, nx2, xf2, _ = dg.dgal_iou_paired(p1, p2)
    assert (host(nx) == host(nx2)).all() and (host(xf) == host(xf2)).all()
    g = np.linspace(-1.0, 2.0, n).astype(np.float32)
    g1, gz1, g2, gz2 = dg.dgal_iou3d_backward(p1, z1, p2, z2, dev(g), nx, xf)
    r1, rz1, r2, rz2 = orc.iou3d_backward_paired(d["p1"], d["p2"], d["z1"], d["z2"], g.astype(np.float64), ref["nx"],
                                                 ref["xflags"], threads=THREADS)
    G = np.concatenate([host(g1), host(g2)], 1)
    R = np.concatenate([r1, r2], 1)
    GZ = np.concatenate([host(gz1), host(gz2)], 1)
    RZ = np.concatenate([rz1, rz2], 1)
    # pairs whose vertical overlap is within rounding of an interval end take
    # a one-sided derivative on either side; compare the rest
    z = d["z1"].astype(np.float64), d["z2"].astype(np.float64)
    ends = np.stack([z[0][:, 0] - z[0][:, 1] / 2, z[0][:, 0] + z[0][:, 1] / 2,
                     z[1][:, 0] - z[1][:, 1] / 2, z[1][:, 0] + z[1][:, 1] / 2], 1)
    tie = (np.abs(ends[:, 1] - ends[:, 3]) < 1e-5) | (np.abs(ends[:, 0] - ends[:, 2]) < 1e-5) | \
          (np.abs(ref["ov"]) < 1e-5)
    rel = _zrel(GZ, RZ, G, R, gen & ~tie)
    assert rel.max() <= GRAD_RTOL, rel.max()


def test_iou3d_equal_extents_is_2d_iou(dg):
    import torch

    d = W.loss_pairs_1m(seed=9, n=50_000)
    p1, p2 = dev(d["p1"]), dev(d["p2"])
    z = torch.stack([torch.linspace(-1, 1, 50_000, device="cuda"), torch.full((50_000,), 1.6, device="cuda")], 1)
    i3, _, _, _ = dg.dgal_iou3d_paired(p1, z.contiguous(), p2, z.contiguous())
    i2, _, _, _ = dg.dgal_iou_paired(p1, p2)
    assert (i3 - i2).abs().max().item() <= 2e-6
    zf = z.clone()
    zf[:, 0] += 5.0
    i0, nx, xf, _ = dg.dgal_iou3d_paired(p1, z.contiguous(), p2, zf.contiguous())
    assert i0.abs().max().item() == 0.0
    g = dg.dgal_iou3d_backward(p1, z.contiguous(), p2, zf.contiguous(), torch.ones(50_000, device="cuda"), nx, xf)
    assert max(t.abs().max().item() for t in g) == 0.0


def test_iou3d_k8_counts_and_loss(dg, orc):
    import torch

    d = W.convex_pairs_4m(seed=6, n=40_000)
    n = d["p1"].shape[0]
    r = np.random.default_rng(10)
    z1 = np.stack([r.uniform(-1, 1, n), r.uniform(1, 2, n)], 1).astype(np.float32)
    z2 = np.stack([z1[:, 0] + r.normal(0, 0.3, n), z1[:, 1] * r.uniform(0.7, 1.3, n)], 1).astype(np.float32)
    p1, p2, c1, c2 = dev(d["p1"]), dev(d["p2"]), dev(d["c1"]), dev(d["c2"])
    Z1, Z2 = dev(z1), dev(z2)
    iou, nx, xf, degen = dg.dgal_iou3d_paired(p1, Z1, p2, Z2, c1, c2, with_degen=True)
    ref = orc.iou3d_paired(d["p1"], d["p2"], z1, z2, d["c1"], d["c2"], threads=THREADS)
    assert np.abs(host(iou) - ref["iou"]).max() <= IOU_ATOL
    w = np.linspace(0.5, 1.5, n).astype(np.float32)
    loss, g1, gz1, g2, gz2, iv = dg.dgal_iou3d_loss(p1, Z1, p2, Z2, dev(w), 0.5, c1, c2, with_iou=True)
    assert torch.equal(iv, iou)
    ref_loss = 0.5 * float(np.sum(w.astype(np.float64) * (1.0 - ref["iou"])))
    assert abs(host(loss)[0] - ref_loss) <= IOU_ATOL * 0.5 * np.abs(w).sum() + 1e-6 * abs(ref_loss)
    b = dg.dgal_iou3d_backward(p1, Z1, p2, Z2, -0.5 * dev(w), nx, xf, c1, c2)
    for u, v in zip(b, (g1, gz1, g2, gz2)):
        assert torch.equal(u, v)
    # autograd wrapper: mean reduction
    P1 = p1.clone().requires_grad_(True)
    ZZ1 = Z1.clone().requires_grad_(True)
    L = dg.iou3d_loss(P1, ZZ1, p2, Z2, c1=c1, c2=c2, reduction="mean")
    L.backward()
    _, h1, hz1, _, _, _ = dg.dgal_iou3d_loss(p1, Z1, p2, Z2, None, 1.0 / n, c1, c2)
    assert torch.allclose(P1.grad, h1, rtol=1e-6, atol=0) and torch.allclose(ZZ1.grad, hz1, rtol=1e-6, atol=0)
