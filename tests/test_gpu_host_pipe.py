"""dgal_iou_fwd_bwd_host (paired forward + backward on host buffers) gives
bit-identical results to the device-memory calls in both of its forms: the
direct kernel on pinned buffers, and the chunked pipeline (pageable buffers),
for ragged chunk tails, one chunk, tiny and empty inputs; and a sample agrees
with the FP64 oracle."""
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


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("n,chunk", [(300_007, 65_536), (50_000, 131_072), (1, 1000), (7, 3)])
def test_host_pipeline_matches_device_path(dg, n, chunk, pinned):
    import torch

    d = W.loss_pairs_1m(seed=40, n=n)
    r = np.random.default_rng(41)
    grad = r.normal(size=n).astype(np.float32)
    hp1 = torch.from_numpy(d["p1"])
    hp2 = torch.from_numpy(d["p2"])
    hg = torch.from_numpy(grad)
    if pinned:  # the direct form
        hp1, hp2, hg = hp1.pin_memory(), hp2.pin_memory(), hg.pin_memory()
    iou, g1, g2 = dg.dgal_iou_fwd_bwd_host(hp1, hp2, hg, chunk=chunk)
    torch.cuda.synchronize()
    p1, p2, gd = dev(d["p1"]), dev(d["p2"]), dev(grad)
    ri, rnx, rxf, _ = dg.dgal_iou_paired(p1, p2)
    r1, r2 = dg.dgal_iou_backward(p1, p2, gd, rnx, rxf)
    torch.cuda.synchronize()
    if n >= dg.dgal_get_paired_config(4)["group_below"] or not pinned:
        assert np.array_equal(iou.numpy(), host(ri))
        assert np.array_equal(g1.numpy(), host(r1)) and np.array_equal(g2.numpy(), host(r2))
    else:
        # a batch this small takes 8-lane groups on the device and one lane
        # per pair in the host-resident kernel: equal up to rounding
        assert np.abs(iou.numpy() - host(ri)).max() <= 1e-6
        m = max(np.abs(host(r1)).max(), np.abs(host(r2)).max(), 1e-30)
        assert np.abs(g1.numpy() - host(r1)).max() <= 1e-5 * m and np.abs(g2.numpy() - host(r2)).max() <= 1e-5 * m
    assert dg.dgal_get_device_status() == 0


@pytest.mark.parametrize("pinned", [True, False])
@pytest.mark.parametrize("K,n,chunk", [(8, 100_003, 32_768), (8, 5, 2), (4, 30_001, 8_192)])
def test_host_pipeline_counts_matches_device_path(dg, K, n, chunk, pinned):
    """General convex polygons with vertex counts (K = 8: constructed
    degenerate pairs included, always staged; K = 4: triangles and
    quadrilaterals, the direct form when pinned) through the host call."""
    import torch

    d = W.convex_pairs_4m(seed=43, n=n, K=K, degenerate_frac=0.05 if K == 8 else 0.0)
    r = np.random.default_rng(44)
    grad = r.normal(size=n).astype(np.float32)
    hp1, hp2 = torch.from_numpy(d["p1"]), torch.from_numpy(d["p2"])
    hc1, hc2 = torch.from_numpy(d["c1"]), torch.from_numpy(d["c2"])
    hg = torch.from_numpy(grad)
    if pinned:
        hp1, hp2, hc1, hc2, hg = (t.pin_memory() for t in (hp1, hp2, hc1, hc2, hg))
    iou, g1, g2 = dg.dgal_iou_fwd_bwd_host(hp1, hp2, hg, c1=hc1, c2=hc2, chunk=chunk)
    torch.cuda.synchronize()
    p1, p2, c1, c2, gd = dev(d["p1"]), dev(d["p2"]), dev(d["c1"]), dev(d["c2"]), dev(grad)
    ri, rnx, rxf, _ = dg.dgal_iou_paired(p1, p2, c1, c2)
    r1, r2 = dg.dgal_iou_backward(p1, p2, gd, rnx, rxf, c1, c2)
    torch.cuda.synchronize()
    assert np.array_equal(iou.numpy(), host(ri))
    assert np.array_equal(g1.numpy(), host(r1)) and np.array_equal(g2.numpy(), host(r2))
    assert dg.dgal_get_device_status() == 0


def test_host_pipeline_unaligned_pinned_views_take_the_staged_form(dg):
    """Pinned buffers whose polygon views start 4 bytes into an allocation
    cannot take the direct form's 16-byte vertex loads: the call stages them,
    with the same results."""
    import torch

    n = 10_001
    d = W.loss_pairs_1m(seed=45, n=n)
    flat1 = torch.empty(n * 8 + 1).pin_memory()
    flat2 = torch.empty(n * 8 + 1).pin_memory()
    hp1 = flat1[1:].view(n, 4, 2)
    hp2 = flat2[1:].view(n, 4, 2)
    hp1.copy_(torch.from_numpy(d["p1"]))
    hp2.copy_(torch.from_numpy(d["p2"]))
    assert hp1.data_ptr() % 16 != 0
    hg = torch.ones(n).pin_memory()
    iou, g1, g2 = dg.dgal_iou_fwd_bwd_host(hp1, hp2, hg, chunk=4096)
    torch.cuda.synchronize()
    p1, p2 = dev(d["p1"]), dev(d["p2"])
    ri, rnx, rxf, _ = dg.dgal_iou_paired(p1, p2)
    r1, r2 = dg.dgal_iou_backward(p1, p2, dev(np.ones(n, np.float32)), rnx, rxf)
    torch.cuda.synchronize()
    assert np.array_equal(iou.numpy(), host(ri))
    assert np.array_equal(g1.numpy(), host(r1)) and np.array_equal(g2.numpy(), host(r2))


def test_host_pipeline_oracle_sample_and_edges(dg, orc):
    import torch

    n = 20_000
    d = W.loss_pairs_1m(seed=42, n=n)
    hp1 = torch.from_numpy(d["p1"]).pin_memory()
    hp2 = torch.from_numpy(d["p2"]).pin_memory()
    hg = torch.ones(n).pin_memory()
    iou, g1, g2 = dg.dgal_iou_fwd_bwd_host(hp1, hp2, hg, chunk=4096)
    torch.cuda.synchronize()
    ref = orc.iou_paired(d["p1"], d["p2"], threads=THREADS)
    assert np.abs(iou.numpy().astype(np.float64) - ref["iou"]).max() <= IOU_ATOL
    o1, o2 = orc.iou_backward_paired(d["p1"], d["p2"], np.ones(n), ref["nx"], ref["xflags"], threads=THREADS)
    rel = grad_rel_err(g1.numpy(), g2.numpy(), o1, o2, ref["degen"] == 0)
    assert rel.max() <= GRAD_RTOL
    # empty input: nothing to do
    z = torch.empty((0, 4, 2)).pin_memory()
    out = dg.dgal_iou_fwd_bwd_host(z, z, torch.empty(0).pin_memory())
    assert out[0].numel() == 0
    # the staged form (pageable buffers) rejects a workspace too small on the host
    ws = torch.empty(1024, device="cuda", dtype=torch.uint8)
    with pytest.raises(dg.DgalError):
        dg.dgal_iou_fwd_bwd_host(torch.from_numpy(d["p1"]), torch.from_numpy(d["p2"]), torch.ones(n), chunk=4096,
                                 workspace=ws)
