"""GPU parity of the pairwise matrix and the ragged batch against the oracle."""
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


def _check_matrix(iou, nx, ref_iou, ref_nx, label):
    err = np.abs(iou.astype(np.float64) - ref_iou)
    assert err.max() <= IOU_ATOL, f"{label}: max IoU err {err.max():.3e}"
    # nx is compared where the oracle's pair is not near-degenerate; the
    # matrix carries no degeneracy byte, so any mismatch must be a pair the
    # paired oracle flags
    return np.nonzero(nx != ref_nx)


def _assert_flagged(orc, a, b, rows, cols, ca=None, cb=None, label=""):
    """Every (row, col) entry whose nx differs from the oracle's must be a pair
    the oracle classifies near-degenerate."""
    if len(rows) == 0:
        return
    o = orc.iou_paired(a[rows], b[cols], None if ca is None else ca[rows], None if cb is None else cb[cols])
    bad = np.nonzero(o["degen"] == 0)[0]
    assert bad.size == 0, f"{label}: nx differs on {bad.size} pairs the oracle does not flag, first {bad[:5]}"


def test_pairwise_bev_full(dg, orc):
    """The 2000 x 2000 bird's-eye matrix, every entry."""
    d = W.pairwise_bev_2000(seed=0)
    iou, nx = dg.dgal_iou_pairwise(dev(d["a"]), dev(d["b"]))
    ref_iou, ref_nx = orc.iou_pairwise(d["a"], d["b"], threads=THREADS)
    bad = _check_matrix(host(iou), host(nx), ref_iou, ref_nx, "pairwise 2000x2000")
    _assert_flagged(orc, d["a"], d["b"], bad[0], bad[1], label="pairwise 2000x2000")
    assert (ref_iou > 0).mean() > 0.001  # the workload has overlaps


@pytest.mark.parametrize("N,M", [(257, 129), (1, 1), (3, 1000), (1000, 3)])
def test_pairwise_ragged_shapes(dg, orc, N, M):
    d = W.pairwise_bev_2000(seed=N + M, N=N, M=M)
    iou, nx = dg.dgal_iou_pairwise(dev(d["a"]), dev(d["b"]))
    ref_iou, ref_nx = orc.iou_pairwise(d["a"], d["b"])
    bad = _check_matrix(host(iou), host(nx), ref_iou, ref_nx, f"pairwise {N}x{M}")
    _assert_flagged(orc, d["a"], d["b"], bad[0], bad[1], label=f"pairwise {N}x{M}")


def test_pairwise_k8_counts(dg, orc):
    d = W.convex_pairs_4m(seed=3, n=600, degenerate_frac=0.0)
    a, b, ca, cb = d["p1"][:300], d["p2"][300:], d["c1"][:300], d["c2"][300:]
    iou, nx = dg.dgal_iou_pairwise(dev(a), dev(b), dev(ca), dev(cb))
    ref_iou, ref_nx = orc.iou_pairwise(a, b, ca, cb)
    bad = _check_matrix(host(iou), host(nx), ref_iou, ref_nx, "pairwise K=8")
    _assert_flagged(orc, a, b, bad[0], bad[1], ca, cb, label="pairwise K=8")


def _batched_inputs(seed=0, S=64):
    d = W.ragged_scenes_64(seed=seed, S=S)
    return d, dev(d["a"]), dev(d["b"]), dev(d["a_off"]), dev(d["b_off"]), dev(d["out_off"])


def _oracle_batched(orc, d):
    S = len(d["N"])
    iou = np.zeros(int(d["out_off"][-1]))
    nx = np.zeros(int(d["out_off"][-1]), np.uint8)
    for s in range(S):
        a = d["a"][d["a_off"][s]:d["a_off"][s + 1]]
        b = d["b"][d["b_off"][s]:d["b_off"][s + 1]]
        r, n = orc.iou_pairwise(a, b, threads=THREADS)
        iou[d["out_off"][s]:d["out_off"][s + 1]] = r.ravel()
        nx[d["out_off"][s]:d["out_off"][s + 1]] = n.ravel()
    return iou, nx


def test_batched_ragged_full(dg, orc):
    """64 ragged scenes (~1e7 entries) in one persistent launch, every entry."""
    d, a, b, ao, bo, oo = _batched_inputs()
    total = int(d["out_off"][-1])
    iou, nx = dg.dgal_iou_pairwise_batched(a, b, ao, bo, oo, total=total)
    ref_iou, ref_nx = _oracle_batched(orc, d)
    err = np.abs(host(iou).astype(np.float64) - ref_iou)
    assert err.max() <= IOU_ATOL
    # every nx mismatch is an entry whose pair the oracle flags near-degenerate
    ent = np.nonzero(host(nx) != ref_nx)[0]
    scene = np.searchsorted(d["out_off"], ent, side="right") - 1
    loc = ent - d["out_off"][scene]
    rows = d["a_off"][scene] + loc // d["M"][scene]
    cols = d["b_off"][scene] + loc % d["M"][scene]
    _assert_flagged(orc, d["a"], d["b"], rows, cols, label="ragged batch")
    # the plain per-scene form and the CUDA-graph form give identical bytes
    iou2, nx2 = dg.dgal_iou_pairwise_per_scene(a, b, d["a_off"], d["b_off"], d["out_off"],
                                               flags=dg.DGAL_FP64_REFINE)
    g = dg.BatchedGraph(a, b, ao, bo, oo, total)
    iou3, nx3 = g.launch()
    import torch

    torch.cuda.synchronize()
    assert torch.equal(iou, iou2) and torch.equal(nx, nx2)
    assert torch.equal(iou, iou3) and torch.equal(nx, nx3)
    # replay after rewriting the inputs in place
    a.copy_(torch.flip(a, [0]))
    iou4, _ = dg.dgal_iou_pairwise_batched(a, b, ao, bo, oo, total=total)
    g.launch()
    torch.cuda.synchronize()
    assert torch.equal(g.iou, iou4)
    g.close()
    assert dg.dgal_get_device_status() == 0


def test_batched_empty_scenes_and_tiles(dg, orc):
    """Scenes with N = 0 or M = 0, and every autotuner tile shape."""
    import torch

    d = W.ragged_scenes_64(seed=5, S=6, n_range=(0, 40), m_range=(0, 7))
    a, b = dev(d["a"]), dev(d["b"])
    ao, bo, oo = dev(d["a_off"]), dev(d["b_off"]), dev(d["out_off"])
    total = int(d["out_off"][-1])
    ref_iou, _ = _oracle_batched(orc, d)
    iou, _ = dg.dgal_iou_pairwise_batched(a, b, ao, bo, oo, total=total)
    assert np.abs(host(iou) - ref_iou).max() <= IOU_ATOL
    # S = 0 is a no-op
    e = torch.zeros(1, dtype=torch.int64, device="cuda")
    dg.dgal_iou_pairwise_batched(a, b, e, e, e, total=0)


def test_batched_bad_offsets_flagged(dg):
    import torch

    d = W.ragged_scenes_64(seed=6, S=4, n_range=(5, 9), m_range=(5, 9))
    oo = d["out_off"].copy()
    oo[2:] += 1  # scene 1 claims one entry too many
    dg.dgal_get_device_status(clear=True)
    dg.dgal_iou_pairwise_batched(dev(d["a"]), dev(d["b"]), dev(d["a_off"]), dev(d["b_off"]), dev(oo),
                                 total=int(oo[-1]))
    torch.cuda.synchronize()
    assert dg.dgal_get_device_status(clear=True) & dg.DGAL_DEV_BAD_OFFSETS


def test_autotune_cache(dg, tmp_path):
    path = tmp_path / "tune.json"
    cfg = dg.dgal_autotune(4, cache_path=path)
    assert cfg["tile"] > 0 and cfg["threads"] in (128, 256)
    text = path.read_text()
    assert "K=4" in text
    # a second call reads the cache
    assert dg.dgal_autotune(4, cache_path=path) == cfg


def test_autotune_cache_rejects_invalid_shapes(dg, tmp_path):
    """A cached shape the ragged kernel cannot take (512 threads: the queue
    codes hold the column in 8 bits) is ignored and the shape tuned again."""
    path = tmp_path / "tune.json"
    cfg = dg.dgal_autotune(4, cache_path=path)
    text = path.read_text()
    key = text.split('"')[1]
    path.write_text('{\n  "%s": [4096, 512, 4]\n}\n' % key)
    again = dg.dgal_autotune(4, cache_path=path)
    assert again["threads"] in (128, 256) and again["threads"] * again["blocks_per_sm"] <= 2048
    assert ", 512," not in path.read_text()
    assert dg.dgal_get_device_status() == 0
