"""GPU parity of the paired forward / backward against the FP64 oracle."""
import numpy as np
import pytest

from paper_2011_11134_gb300 import workloads as W

from .gpu_helpers import GRAD_RTOL, IOU_ATOL, THREADS, check_flagged_grads, check_forward, dev, grad_rel_err, host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_11134_gb300 as m

    m.dgal_get_device_status(clear=True)
    return m


def _fwd(dg, p1, p2, c1=None, c2=None, flags=None):
    kw = {} if flags is None else dict(flags=flags)
    iou, nx, xf, degen = dg.dgal_iou_paired(dev(p1), dev(p2), None if c1 is None else dev(c1),
                                            None if c2 is None else dev(c2), with_degen=True, **kw)
    return host(iou), host(nx), host(xf), host(degen)


@pytest.mark.parametrize("n", [4096, 4096 + 37, 1])
def test_paired_rect_forward(dg, orc, n):
    d = W.paired_rect_4096(seed=0, n=n)
    iou, nx, xf, degen = _fwd(dg, d["p1"], d["p2"])
    ref = orc.iou_paired(d["p1"], d["p2"], threads=THREADS)
    gen = check_forward(iou, nx, xf, degen, ref, "paired K=4")
    assert gen.mean() > 0.99 or n < 10
    assert dg.dgal_get_device_status() == 0


def test_paired_rect_backward_saved_and_recompute(dg, orc):
    import torch

    d = W.paired_rect_4096(seed=0)
    n = d["p1"].shape[0]
    p1, p2 = dev(d["p1"]), dev(d["p2"])
    grad = torch.from_numpy(np.linspace(-1.5, 2.0, n).astype(np.float32)).cuda()
    iou, nx, xf, degen = dg.dgal_iou_paired(p1, p2, with_degen=True)
    g1, g2 = dg.dgal_iou_backward(p1, p2, grad, nx, xf)
    r1, r2 = dg.dgal_iou_backward(p1, p2, grad)  # recompute
    ref = orc.iou_paired(d["p1"], d["p2"])
    o1, o2 = orc.iou_backward_paired(d["p1"], d["p2"], host(grad).astype(np.float64), ref["nx"], ref["xflags"])
    gen = (ref["degen"] == 0) & ((host(degen) & 1) == 0)
    rel = grad_rel_err(host(g1), host(g2), o1, o2, gen)
    assert rel.max() <= GRAD_RTOL, f"saved-flag grads: max rel err {rel.max():.3e}"
    # recompute mode agrees with the saved-flag gradients (identical arithmetic
    # on generic pairs; near-degenerate pairs may take the shoelace adjoint in
    # one mode and the shape derivative in the other)
    scale = max(g1.abs().max().item(), g2.abs().max().item())
    assert (g1 - r1).abs().max().item() <= 1e-5 * scale and (g2 - r2).abs().max().item() <= 1e-5 * scale
    same = torch.from_numpy(gen).cuda()
    assert torch.equal(g1[same], r1[same]) and torch.equal(g2[same], r2[same])


def test_loss_pairs_full_size(dg, orc):
    """The 1M-pair IoU-loss workload, forward + backward on every pair."""
    import torch

    d = W.loss_pairs_1m(seed=0)
    p1, p2 = dev(d["p1"]), dev(d["p2"])
    grad = torch.ones(p1.shape[0], device="cuda")
    iou, nx, xf, degen = dg.dgal_iou_paired(p1, p2, with_degen=True)
    g1, g2 = dg.dgal_iou_backward(p1, p2, grad, nx, xf)
    ref = orc.iou_paired(d["p1"], d["p2"], threads=THREADS)
    gen = check_forward(host(iou), host(nx), host(xf), host(degen), ref, "loss 1M")
    o1, o2 = orc.iou_backward_paired(d["p1"], d["p2"], np.ones(p1.shape[0]), ref["nx"], ref["xflags"],
                                     threads=THREADS)
    rel = grad_rel_err(host(g1), host(g2), o1, o2, gen)
    assert rel.max() <= GRAD_RTOL, f"1M grads: max rel err {rel.max():.3e} at {int(rel.argmax())}"
    check_flagged_grads(host(g1), host(g2), d["p1"], d["p2"], None, None, ref, ~gen, label="loss 1M")
    # pairs whose small orientations took the FP64 definition's sign (degen
    # bit 1) keep the definition's combinatorics: nx and xflags as the oracle's
    rep = (host(degen) & 2) != 0
    assert rep.sum() > 100, "the workload has near-degenerate pairs"
    assert (host(nx)[rep] == ref["nx"][rep]).all()
    assert (host(xf)[rep] == ref["xflags"][rep]).all()


def test_finite_differences_1000(dg, orc):
    """GPU gradients vs central differences of the FP64 oracle on 1000 pairs."""
    d = W.loss_pairs_1m(seed=0, n=1000)
    p1, p2 = dev(d["p1"]), dev(d["p2"])
    import torch

    iou, nx, xf, degen = dg.dgal_iou_paired(p1, p2, with_degen=True)
    g1, g2 = dg.dgal_iou_backward(p1, p2, torch.ones(1000, device="cuda"), nx, xf)
    g1, g2, degen = host(g1), host(g2), host(degen)
    checked = 0
    for k in range(1000):
        P, Q = d["p1"][k].astype(np.float64), d["p2"][k].astype(np.float64)
        base = orc.iou_pair_f64(P, Q, 4)
        if base[6] or (degen[k] & 1) or base[4] == 0:
            continue
        L = max(np.abs(P - P[0]).max(), np.abs(Q - P[0]).max())
        h = 1e-6 * L
        num = np.zeros((2, 4, 2))
        ok = True
        for w in range(2):
            for v in range(4):
                for c in range(2):
                    vals = []
                    for sg in (1, -1):
                        A, B = P.copy(), Q.copy()
                        (A if w == 0 else B)[v, c] += sg * h
                        r = orc.iou_pair_f64(A, B, 4)
                        ok &= r[4] == base[4] and list(r[5]) == list(base[5])
                        vals.append(r[0])
                    num[w, v, c] = (vals[0] - vals[1]) / (2 * h)
        if not ok:
            continue
        G = np.stack([g1[k], g2[k]]).astype(np.float64)
        rel = np.abs(G - num).max() / max(np.abs(num).max(), 1e-6)
        assert rel <= GRAD_RTOL, f"pair {k}: FD rel err {rel:.3e}"
        checked += 1
    assert checked >= 900


def test_autograd_function(dg):
    import torch

    d = W.paired_rect_4096(seed=2, n=777)
    p1 = dev(d["p1"]).requires_grad_(True)
    p2 = dev(d["p2"]).requires_grad_(True)
    w = torch.rand(777, device="cuda")
    (dg.iou(p1, p2) * w).sum().backward()
    a1, a2 = p1.grad.clone(), p2.grad.clone()
    p1.grad = None
    p2.grad = None
    (dg.iou(p1, p2, recompute=True) * w).sum().backward()
    scale = max(a1.abs().max().item(), a2.abs().max().item())
    assert (a1 - p1.grad).abs().max().item() <= 1e-5 * scale and (a2 - p2.grad).abs().max().item() <= 1e-5 * scale
    _, nx, xf, _ = dg.dgal_iou_paired(p1.detach(), p2.detach())
    b1, b2 = dg.dgal_iou_backward(p1.detach(), p2.detach(), w, nx, xf)
    assert torch.equal(a1, b1) and torch.equal(a2, b2)


def test_convex_k8_with_degenerate(dg, orc):
    """General convex polygons (K=8, counts 3..8) with 5% constructed
    near-degenerate pairs; FP64 refinement on.  IoU within 1e-5 on every
    pair (generic and degenerate), flags exact and grads within 1e-3 on
    generic pairs."""
    import torch

    d = W.convex_pairs_4m(seed=0, n=200_000)
    p1, p2, c1, c2 = dev(d["p1"]), dev(d["p2"]), dev(d["c1"]), dev(d["c2"])
    iou, nx, xf, degen = dg.dgal_iou_paired(p1, p2, c1, c2, with_degen=True)
    ref = orc.iou_paired(d["p1"], d["p2"], d["c1"], d["c2"], threads=THREADS)
    gen = check_forward(host(iou), host(nx), host(xf), host(degen), ref, "convex K=8")
    kind = d["kind"]
    hd = host(degen)
    assert (hd[kind > 0] & 1).all(), "every constructed degenerate pair is flagged"
    # identical pairs are recognised as such; the others take FP64 orientations
    assert (hd[kind > 1] & 2).all(), "and refined in FP64"
    grad = torch.ones(p1.shape[0], device="cuda")
    g1, g2 = dg.dgal_iou_backward(p1, p2, grad, nx, xf, c1, c2)
    o1, o2 = orc.iou_backward_paired(d["p1"], d["p2"], np.ones(p1.shape[0]), ref["nx"], ref["xflags"], d["c1"],
                                     d["c2"], threads=THREADS)
    rel = grad_rel_err(host(g1), host(g2), o1, o2, gen)
    assert rel.max() <= GRAD_RTOL, f"K=8 grads: max rel err {rel.max():.3e} at {int(np.nonzero(gen)[0][rel.argmax()])}"
    check_flagged_grads(host(g1), host(g2), d["p1"], d["p2"], d["c1"], d["c2"], ref, ~gen, label="convex K=8")
    # padded slots get exactly zero gradient
    cnt1 = d["c1"].astype(int)
    pad = np.arange(8)[None, :] >= cnt1[:, None]
    assert (host(g1)[pad] == 0).all()
    assert dg.dgal_get_device_status() == 0


def test_convex_k8_full_size_sampled(dg, orc):
    """The 4M-pair convex workload at full size, in the bench's launch
    configuration (forward saving flags, backward from them), checked on a
    sample the oracle computes pair by pair: 20,000 random pairs plus 2,000
    constructed near-degenerate ones."""
    import torch

    d = W.convex_pairs_4m(seed=0)
    n = d["p1"].shape[0]
    p1, p2, c1, c2 = dev(d["p1"]), dev(d["p2"]), dev(d["c1"]), dev(d["c2"])
    iou, nx, xf, degen = dg.dgal_iou_paired(p1, p2, c1, c2, with_degen=True)
    g1, g2 = dg.dgal_iou_backward(p1, p2, torch.ones(n, device="cuda"), nx, xf, c1, c2)
    torch.cuda.synchronize()
    assert dg.dgal_get_device_status() == 0
    rng = np.random.default_rng(11)
    idx = np.union1d(rng.choice(n, 20_000, replace=False), rng.choice(np.flatnonzero(d["kind"] > 0), 2_000,
                                                                      replace=False))
    s1, s2, sc1, sc2 = d["p1"][idx], d["p2"][idx], d["c1"][idx], d["c2"][idx]
    ref = orc.iou_paired(s1, s2, sc1, sc2, threads=THREADS)
    gen = check_forward(host(iou)[idx], host(nx)[idx], host(xf)[idx], host(degen)[idx], ref, "convex 4M sample")
    o1, o2 = orc.iou_backward_paired(s1, s2, np.ones(len(idx)), ref["nx"], ref["xflags"], sc1, sc2,
                                     threads=THREADS)
    rel = grad_rel_err(host(g1)[idx], host(g2)[idx], o1, o2, gen)
    assert rel.max() <= GRAD_RTOL, f"convex 4M sample grads: max rel err {rel.max():.3e}"
    check_flagged_grads(host(g1)[idx], host(g2)[idx], s1, s2, sc1, sc2, ref, ~gen, label="convex 4M sample")


def test_plain_form_generic_parity(dg, orc):
    """DGAL_PLAIN (FP32 only, recompute backward) matches on generic pairs."""
    d = W.paired_rect_4096(seed=4)
    iou, nx, xf, degen = _fwd(dg, d["p1"], d["p2"], flags=dg.DGAL_PLAIN)
    ref = orc.iou_paired(d["p1"], d["p2"])
    check_forward(iou, nx, xf, degen, ref, "plain")


def test_edge_cases(dg, orc):
    import torch

    # empty batch: no launch, empty outputs
    z = torch.zeros((0, 4, 2), device="cuda")
    iou, nx, xf, _ = dg.dgal_iou_paired(z, z)
    assert iou.shape == (0,)
    g1, g2 = dg.dgal_iou_backward(z, z, torch.zeros(0, device="cuda"), nx, xf)
    assert g1.shape == (0, 4, 2)
    # identical, disjoint, nested
    d = W.paired_rect_4096(seed=9, n=300)
    same, _, _, _ = _fwd(dg, d["p1"], d["p1"])
    assert np.abs(same - 1).max() <= 1e-6
    far = d["p2"] + np.float32(100.0)
    sep, nxs, xfs, _ = _fwd(dg, d["p1"], far)
    assert (sep == 0).all() and (nxs == 0).all() and (xfs == 0xFF).all()


def test_bad_counts_set_status(dg):
    import torch

    d = W.convex_pairs_4m(seed=1, n=64, degenerate_frac=0)
    c1 = d["c1"].copy()
    c1[5] = 2
    c1[9] = 9
    dg.dgal_get_device_status(clear=True)
    iou, nx, xf, _ = dg.dgal_iou_paired(dev(d["p1"]), dev(d["p2"]), dev(c1), dev(d["c2"]))
    st = dg.dgal_get_device_status(clear=True)
    assert st & dg.DGAL_DEV_BAD_COUNT
    h = host(iou)
    assert h[5] == 0 and h[9] == 0 and host(nx)[5] == 0
    # corrupted flags in the backward are detected, gradients zeroed, no fault
    xf2 = xf.clone()
    nx2 = nx.clone()
    xf2[0, 0] = 0xC1  # no such code kind
    nx2[1] = 17        # more than 2K vertices
    g1, g2 = dg.dgal_iou_backward(dev(d["p1"]), dev(d["p2"]), torch.ones(64, device="cuda"), nx2, xf2,
                                  dev(d["c1"]), dev(d["c2"]))
    st = dg.dgal_get_device_status(clear=True)
    assert st & dg.DGAL_DEV_BAD_FLAGS
    assert (host(g1)[0] == 0).all() and (host(g1)[1] == 0).all()


def test_thin_pairs_within_tolerance(dg, orc):
    """Thin rectangles (aspect up to 800) with slightly shifted partners:
    their union is a small fraction of the pair's squared coordinate scale,
    where FP32 shoelace sums lose digits; the IoU stays within 1e-5 of the
    FP64 oracle on every pair, K = 4 paired and pairwise, and K = 8."""
    r = np.random.default_rng(61)
    n = 20000
    c = r.uniform(0, 10, (n, 2))
    w, h = r.uniform(2.0, 4.0, n), r.uniform(0.005, 0.02, n)
    th = r.uniform(-np.pi, np.pi, n)
    p1 = W.boxes_to_polygons(c[:, 0], c[:, 1], w, h, th)
    shift = r.normal(0, 0.004, (n, 2))
    p2 = W.boxes_to_polygons(c[:, 0] + shift[:, 0], c[:, 1] + shift[:, 1], w * r.uniform(0.98, 1.02, n),
                             h * r.uniform(0.8, 1.2, n), th + r.normal(0, 1e-3, n))
    ref = orc.iou_paired(p1, p2, threads=THREADS)
    assert (ref["nx"] >= 3).mean() > 0.5
    iou, _, _, _ = dg.dgal_iou_paired(dev(p1), dev(p2))
    assert np.abs(host(iou).astype(np.float64) - ref["iou"]).max() <= IOU_ATOL
    m, _ = dg.dgal_iou_pairwise(dev(p1[:300]), dev(p2[:300]), with_nx=False)
    rm, _ = orc.iou_pairwise(p1[:300], p2[:300], threads=THREADS)
    assert np.abs(host(m).astype(np.float64) - rm).max() <= IOU_ATOL
    # K = 8: the same rectangles padded with counts
    q1 = np.concatenate([p1, np.repeat(p1[:, :1], 4, 1)], 1).astype(np.float32)
    q2 = np.concatenate([p2, np.repeat(p2[:, :1], 4, 1)], 1).astype(np.float32)
    cnt = np.full(n, 4, np.uint8)
    i8, _, _, _ = dg.dgal_iou_paired(dev(q1), dev(q2), dev(cnt), dev(cnt))
    assert np.abs(host(i8).astype(np.float64) - ref["iou"]).max() <= IOU_ATOL


def test_k4_with_counts(dg, orc):
    """Triangles and quadrilaterals in K = 4 storage (counts 3 or 4): the
    K = 4 kernels' count-aware instantiations, forward, backward from saved
    flags and recomputed, and the pairwise matrix."""
    import torch

    d = W.convex_pairs_4m(seed=17, n=30_000, K=4, degenerate_frac=0.0)
    assert (d["c1"] == 3).any() and (d["c1"] == 4).any()
    p1, p2, c1, c2 = d["p1"], d["p2"], d["c1"], d["c2"]
    iou, nx, xf, degen = _fwd(dg, p1, p2, c1, c2)
    ref = orc.iou_paired(p1, p2, c1, c2, threads=THREADS)
    gen = check_forward(iou, nx, xf, degen, ref, "K=4 counts")
    g = np.ones(p1.shape[0], np.float32)
    r1, r2 = orc.iou_backward_paired(p1, p2, np.ones(p1.shape[0]), ref["nx"], ref["xflags"], c1, c2,
                                     threads=THREADS)
    P1, P2, C1, C2 = dev(p1), dev(p2), dev(c1), dev(c2)
    for saved in (True, False):
        a, b = (dev(nx), dev(xf)) if saved else (None, None)
        g1, g2 = dg.dgal_iou_backward(P1, P2, dev(g), a, b, c1=C1, c2=C2)
        torch.cuda.synchronize()
        rel = grad_rel_err(host(g1), host(g2), r1, r2, gen)
        assert rel.max() <= GRAD_RTOL, (saved, rel.max())
        pad = np.arange(4)[None, :] >= c1.astype(int)[:, None]
        assert (host(g1)[pad] == 0).all()
    m, mnx = dg.dgal_iou_pairwise(P1[:400], P2[:300], C1[:400], C2[:300])
    rm, rnx = orc.iou_pairwise(p1[:400], p2[:300], c1[:400], c2[:300], threads=THREADS)
    assert np.abs(host(m).astype(np.float64) - rm).max() <= IOU_ATOL
    assert dg.dgal_get_device_status() == 0


def test_recompute_chosen_by_flag_budget(dg, monkeypatch):
    """Above the flag budget IoU keeps no flags and its backward re-runs the
    clip; the gradients equal those of the saved-flag mode."""
    import torch

    n = 1000
    d = W.paired_rect_4096(seed=3, n=n)
    w = torch.rand(n, device="cuda")
    grads = []
    for budget, want in ((n * 9 - 1, True), (n * 9, False)):
        p1 = dev(d["p1"]).requires_grad_(True)
        p2 = dev(d["p2"]).requires_grad_(True)
        y = dg.iou(p1, p2, flag_budget=budget)
        assert y.grad_fn.recompute is want
        (y * w).sum().backward()
        grads.append((p1.grad, p2.grad))
    (a1, a2), (b1, b2) = grads
    scale = max(b1.abs().max().item(), b2.abs().max().item())
    assert (a1 - b1).abs().max().item() <= 1e-5 * scale and (a2 - b2).abs().max().item() <= 1e-5 * scale
    # the environment variable sets the default budget
    monkeypatch.setenv("DGAL_FLAG_BUDGET_BYTES", "1")
    assert dg.iou(dev(d["p1"]).requires_grad_(True), dev(d["p2"])).grad_fn.recompute is True


def test_paired_launch_shapes_and_tuner(dg, orc, tmp_path):
    """Both launch shapes of the paired calls (a group of 8 lanes per pair,
    one lane per pair) match the oracle at sizes on either side of the
    threshold, whichever shape the threshold picks; the tuner caches the
    threshold it measures."""
    import torch

    key_dev = None
    for below, sizes in ((1 << 40, (1000, 50_000)), (0, (1000, 50_000))):
        path = tmp_path / f"shape{below}.json"
        if key_dev is None:
            dg.dgal_autotune(4, cache_path=path, config_class=1)
            key_dev = path.read_text().split('"')[1]
            assert key_dev.endswith("|paired")
        path.write_text('{\n  "%s": [%d, 0, 0]\n}\n' % (key_dev, below))
        assert dg.dgal_autotune(4, cache_path=path, config_class=1)["group_below"] == below
        for n in sizes:
            d = W.loss_pairs_1m(seed=31, n=n)
            p1, p2 = dev(d["p1"]), dev(d["p2"])
            iou, nx, xf, degen = dg.dgal_iou_paired(p1, p2, with_degen=True)
            ref = orc.iou_paired(d["p1"], d["p2"], threads=THREADS)
            gen = check_forward(host(iou), host(nx), host(xf), host(degen), ref, f"shape below={below} n={n}")
            grad = torch.linspace(-1, 1, n, device="cuda")
            g1, g2 = dg.dgal_iou_backward(p1, p2, grad, nx, xf)
            r1, r2 = orc.iou_backward_paired(d["p1"], d["p2"], host(grad).astype(np.float64), ref["nx"], ref["xflags"],
                                             threads=THREADS)
            rel = grad_rel_err(host(g1), host(g2), r1, r2, gen)
            assert rel.max() <= GRAD_RTOL, f"below={below} n={n}: {rel.max():.3e}"
            # recompute mode on the same shape
            h1, h2 = dg.dgal_iou_backward(p1, p2, grad)
            m = max(g1.abs().max().item(), g2.abs().max().item())
            assert (h1 - g1).abs().max().item() <= 1e-5 * m
    # a fresh tuning (no cache) leaves a threshold in use
    cfg = dg.dgal_autotune(4, cache_path=tmp_path / "fresh.json", config_class=1)
    assert cfg["group_below"] >= 0
    assert "|paired" in (tmp_path / "fresh.json").read_text()
    assert dg.dgal_get_device_status() == 0
    # back to the untuned threshold for the tests that follow in this process
    path = tmp_path / "default.json"
    path.write_text('{\n  "%s": [1024, 0, 0]\n}\n' % key_dev)
    assert dg.dgal_autotune(4, cache_path=path, config_class=1)["group_below"] == 1024


@pytest.mark.parametrize("K,n", [(4, 4096 + 37), (4, 300), (8, 5003)])
def test_fwd_bwd_one_call(dg, orc, K, n):
    """dgal_iou_fwd_bwd (dL/dIoU given up front): K = 4 in one kernel, K = 8
    through the two kernels with caller scratch; the same values as the two
    separate calls (bit for bit where those take one lane per pair), and the
    oracle's IoU."""
    import ctypes

    import torch

    from paper_2011_11134_gb300 import _lib

    if K == 4:
        d = W.paired_rect_4096(seed=11, n=n)
        c1 = c2 = None
    else:
        d = W.convex_pairs_4m(seed=11, n=n)
        c1, c2 = dev(d["c1"]), dev(d["c2"])
    p1, p2 = dev(d["p1"]), dev(d["p2"])
    grad = torch.linspace(-1.0, 2.0, n, device="cuda")
    iou, g1, g2 = dg.dgal_iou_fwd_bwd(p1, p2, grad, c1, c2)
    ri, rnx, rxf, _ = dg.dgal_iou_paired(p1, p2, c1, c2)
    r1, r2 = dg.dgal_iou_backward(p1, p2, grad, rnx, rxf, c1, c2)
    torch.cuda.synchronize()
    if K == 8 or n >= dg.dgal_get_paired_config(4)["group_below"]:
        assert torch.equal(iou, ri) and torch.equal(g1, r1) and torch.equal(g2, r2)
    else:
        m = max(r1.abs().max().item(), r2.abs().max().item())
        assert (iou - ri).abs().max().item() <= 1e-6
        assert (g1 - r1).abs().max().item() <= 1e-5 * m and (g2 - r2).abs().max().item() <= 1e-5 * m
    f = orc.iou_paired(d["p1"], d["p2"], d.get("c1"), d.get("c2"), threads=THREADS)
    assert np.abs(host(iou) - f["iou"]).max() <= IOU_ATOL
    assert dg.dgal_get_device_status() == 0
    # K = 8 without flag scratch is refused before any launch
    if K == 8:
        lib = _lib.lib()
        st = lib.dgal_iou_fwd_bwd(_lib.ptr(p1), _lib.ptr(c1), _lib.ptr(p2), _lib.ptr(c2), _lib.ptr(grad), n, K,
                                  _lib.ptr(iou), _lib.ptr(g1), _lib.ptr(g2), None, None, dg.DGAL_FP64_REFINE,
                                  _lib.stream_ptr(None))
        assert st != 0 and "scratch" in dg.dgal_last_error()
    # nothing to do
    z = torch.zeros((0, K, 2), device="cuda")
    e = dg.dgal_iou_fwd_bwd(z, z, torch.zeros(0, device="cuda"))
    assert e[0].numel() == 0


def test_forward_backward_in_cuda_graph(dg):
    """The forward and the backward (launched as a programmatic dependent of
    the forward) captured in one CUDA graph and replayed give the eager
    calls' bytes."""
    import torch

    d = W.loss_pairs_1m(seed=4, n=50_000)
    p1, p2 = dev(d["p1"]), dev(d["p2"])
    grad = torch.rand(p1.shape[0], device="cuda")
    iou, nx, xf, _ = dg.dgal_iou_paired(p1, p2)
    g1, g2 = dg.dgal_iou_backward(p1, p2, grad, nx, xf)
    torch.cuda.synchronize()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        dg.dgal_iou_paired(p1, p2)  # warm call on the capture stream
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=s):
            giou, gnx, gxf, _ = dg.dgal_iou_paired(p1, p2)
            h1, h2 = dg.dgal_iou_backward(p1, p2, grad, gnx, gxf)
    torch.cuda.current_stream().wait_stream(s)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(giou, iou) and torch.equal(gnx, nx) and torch.equal(gxf, xf)
    assert torch.equal(h1, g1) and torch.equal(h2, g2)
    assert dg.dgal_get_device_status() == 0


def test_k4_constructed_degenerate(dg, orc):
    """Quadrilaterals and triangles in K = 4 storage with constructed
    near-degenerate partners (identical, shared edge, touching vertex,
    collinear edge 1e-6 off): the one-thread K = 4 kernels, FP64 refinement
    on, where exact zero orientations take their sign from the infinitesimal
    translation of P2.  IoU within 1e-5 on every pair, flags and gradients as
    the oracle's on generic pairs, and bounded gradients on flagged ones."""
    import torch

    d = W.convex_pairs_4m(seed=23, n=40_000, K=4, degenerate_frac=0.5)
    kind = d["kind"]
    assert ((kind == 2) | (kind == 3)).sum() > 5000
    p1, p2, c1, c2 = dev(d["p1"]), dev(d["p2"]), dev(d["c1"]), dev(d["c2"])
    iou, nx, xf, degen = dg.dgal_iou_paired(p1, p2, c1, c2, with_degen=True)
    ref = orc.iou_paired(d["p1"], d["p2"], d["c1"], d["c2"], threads=THREADS)
    gen = check_forward(host(iou), host(nx), host(xf), host(degen), ref, "K=4 degenerate")
    assert (host(degen)[kind > 0] & 1).all(), "every constructed degenerate pair is flagged"
    grad = torch.ones(p1.shape[0], device="cuda")
    g1, g2 = dg.dgal_iou_backward(p1, p2, grad, nx, xf, c1, c2)
    o1, o2 = orc.iou_backward_paired(d["p1"], d["p2"], np.ones(p1.shape[0]), ref["nx"], ref["xflags"], d["c1"],
                                     d["c2"], threads=THREADS)
    rel = grad_rel_err(host(g1), host(g2), o1, o2, gen)
    assert rel.max() <= GRAD_RTOL, f"K=4 grads: max rel err {rel.max():.3e}"
    check_flagged_grads(host(g1), host(g2), d["p1"], d["p2"], d["c1"], d["c2"], ref, ~gen, label="K=4 degenerate")
    assert dg.dgal_get_device_status() == 0
