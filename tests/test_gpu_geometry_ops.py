"""GPU parity of the exported geometry operations (dgal_intersect_paired,
dgal_area, the line operations) against the FP64 oracle.

Tolerances follow from FP32 rounding (u = 2^-24): input vertices are copied
(exact); a crossing vertex a + t (b - a) with t = S / D carries the error of
S (at most about 48 u L^2, L the pair's coordinate scale) divided by |D| and
scaled by |b - a|, plus the rounding of the sum; areas are shoelace sums with
an error of order u L^2 per term."""
import numpy as np
import pytest

from paper_2011_11134_gb300 import workloads as W

from .gpu_helpers import THREADS, dev, host

pytestmark = pytest.mark.gpu
U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def dg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_11134_gb300 as m

    m.dgal_get_device_status(clear=True)
    return m


def _crossing_tol(p1, p2, code, k, n1, n2, L):
    i, j = (code >> 3) & 7, code & 7
    a, b = p1[k, i].astype(np.float64), p1[k, (i + 1) % n1].astype(np.float64)
    c, d = p2[k, j].astype(np.float64), p2[k, (j + 1) % n2].astype(np.float64)
    r, s = b - a, d - c
    D = abs(r[0] * s[1] - r[1] * s[0])
    return 64 * U32 * L * L * np.hypot(*r) / D + 16 * U32 * L


@pytest.mark.parametrize("K", [4, 8])
def test_intersect_vertices_and_area(dg, orc, K):
    if K == 4:
        d = W.loss_pairs_1m(seed=21, n=20000)
        p1, p2, c1, c2 = d["p1"], d["p2"], None, None
    else:
        d = W.convex_pairs_4m(seed=21, n=20000)
        p1, p2, c1, c2 = d["p1"], d["p2"], d["c1"], d["c2"]
    verts, area, nx, xf = dg.dgal_intersect_paired(dev(p1), dev(p2), None if c1 is None else dev(c1),
                                                   None if c2 is None else dev(c2))
    verts, area, nx, xf = host(verts), host(area), host(nx), host(xf)
    ref = orc.intersect_paired(p1, p2, c1, c2, threads=THREADS)
    fw = orc.iou_paired(p1, p2, c1, c2, threads=THREADS)
    gen = fw["degen"] == 0
    assert (nx[gen] == ref["nx"][gen]).all() and (xf[gen] == ref["xflags"][gen]).all()
    o = p1[:, :1, :].astype(np.float64)
    Ls = np.maximum(np.abs(p1 - o).max((1, 2)), np.abs(p2 - o).max((1, 2)))
    # areas: every pair (the area is continuous through degenerate contact)
    aerr = np.abs(area.astype(np.float64) - fw["areas"][:, 0])
    assert (aerr <= 64 * U32 * Ls * Ls * 2 * K).all(), aerr.max()
    checked = 0
    for k in np.nonzero(gen)[0][:4000]:
        n1 = K if c1 is None else int(c1[k])
        n2 = K if c2 is None else int(c2[k])
        m = int(nx[k])
        assert (verts[k, m:] == 0).all()
        for s in range(m):
            code = int(xf[k, s])
            got, want = verts[k, s].astype(np.float64), ref["verts"][k, s]
            if code < 0x80:
                assert (got == want).all(), (k, s)  # input vertex, copied
            else:
                tol = _crossing_tol(p1, p2, code, k, n1, n2, Ls[k])
                assert np.abs(got - want).max() <= tol, (k, s, np.abs(got - want).max(), tol)
        checked += 1
    assert checked > 1000
    assert dg.dgal_get_device_status() == 0


def test_area_parity(dg, orc):
    c = W.convex_pairs_4m(seed=22, n=50000, degenerate_frac=0.0)
    got = host(dg.dgal_area(dev(c["p1"]), dev(c["c1"]))).astype(np.float64)
    want = orc.area(c["p1"], c["c1"])
    L = np.abs(c["p1"] - c["p1"][:, :1]).max((1, 2)).astype(np.float64)
    assert (np.abs(got - want) <= 32 * U32 * L * L * 8).all()
    d = W.paired_rect_4096(seed=22, n=4097)
    got = host(dg.dgal_area(dev(d["p1"]))).astype(np.float64)
    assert np.allclose(got, orc.area(d["p1"]), rtol=1e-5, atol=0)
    bad = c["c1"].copy()
    bad[3] = 1
    assert host(dg.dgal_area(dev(c["p1"]), dev(bad)))[3] == 0
    assert dg.dgal_get_device_status(clear=True) & dg.DGAL_DEV_BAD_COUNT


def test_lines_forward_backward(dg, orc):
    import torch

    r = np.random.default_rng(23)
    n = 100_003
    p, q = r.uniform(-10, 10, (n, 2)).astype(np.float32), r.uniform(-10, 10, (n, 2)).astype(np.float32)
    s_, t_ = r.uniform(-10, 10, (n, 2)).astype(np.float32), r.uniform(-10, 10, (n, 2)).astype(np.float32)
    P, Q, S, T = dev(p), dev(q), dev(s_), dev(t_)
    l1, l2 = dg.dgal_line_from_points(P, Q), dg.dgal_line_from_points(S, T)
    r1 = orc.line_from_points(p, q)
    # a, b: one rounding each; c: two products and a difference
    tolc = 4 * U32 * (np.abs(p[:, 0] * q[:, 1]) + np.abs(q[:, 0] * p[:, 1]))
    e = np.abs(host(l1).astype(np.float64) - r1)
    assert (e[:, :2] <= 2 * U32 * 20).all() and (e[:, 2] <= tolc + 1e-30).all()
    # intersection, on the lines as the GPU rounded them
    L1, L2 = host(l1).astype(np.float64), host(l2).astype(np.float64)
    x = host(dg.dgal_line_intersect(l1, l2)).astype(np.float64)
    xr = orc.line_intersect(L1, L2)
    a1, b1, c1 = L1.T
    a2, b2, c2 = L2.T
    W_ = np.abs(a1 * b2 - a2 * b1)
    cond = (np.abs(b1 * c2) + np.abs(b2 * c1) + np.abs(c1 * a2) + np.abs(c2 * a1)
            + (np.abs(xr).max(1)) * (np.abs(a1 * b2) + np.abs(a2 * b1))) / W_
    ok = W_ > 1e-3 * (np.abs(a1 * b2) + np.abs(a2 * b1))
    assert ok.mean() > 0.99
    assert (np.abs(x - xr).max(1)[ok] <= 8 * U32 * cond[ok]).all()
    # backward through autograd
    Pg, Qg = P.clone().requires_grad_(True), Q.clone().requires_grad_(True)
    g = r.normal(size=(n, 2)).astype(np.float32)
    pt = dg.line_intersect(dg.line_from_points(Pg, Qg), l2)
    pt.backward(dev(g))
    torch.cuda.synchronize()
    gl1, _ = orc.line_intersect_backward(L1, L2, g)
    gp, gq = orc.line_from_points_backward(p, q, gl1)
    okb = ok & (W_ > 1e-1 * (np.abs(a1 * b2) + np.abs(a2 * b1)))
    # each gradient component is a short sum of products (dL/dl1 times a
    # coordinate), which can cancel: the FP32 error is bounded relative to
    # the magnitude of the summed terms, not to the result
    # (dL/dl1 is itself such a sum: gW b2 - gY c2, ... with gX = g_x / W,
    # gY = g_y / W, gW = -(g . x) / W)
    Wsg = a1 * b2 - a2 * b1
    gsum = (np.abs(g).sum(1) * (1.0 + np.abs(xr).sum(1))) / np.abs(Wsg)
    tg = gsum * np.abs(L2).max(1)
    terms = tg * (1.0 + np.maximum(np.abs(p).max(1), np.abs(q).max(1)))
    for got, want in ((host(Pg.grad), gp), (host(Qg.grad), gq)):
        rel = np.abs(got - want).max(1) / terms
        assert rel[okb].max() <= 1e-5, rel[okb].max()
        big = np.abs(want).max(1) >= 1e-2 * terms  # no heavy cancellation
        rel2 = np.abs(got - want).max(1) / np.abs(want).max(1)
        assert rel2[okb & big].max() <= 1e-3, rel2[okb & big].max()
    # parallel lines: non-finite
    par = dg.dgal_line_intersect(dev(np.array([[0, 1, 0]], np.float32)), dev(np.array([[0, 2, 1]], np.float32)))
    assert not torch.isfinite(par).all()
    # empty
    z = torch.empty((0, 2), device="cuda")
    assert dg.dgal_line_from_points(z, z).shape == (0, 3)
