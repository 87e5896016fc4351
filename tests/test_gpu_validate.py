"""The DGAL_VALIDATE input check on the GPU (dgal_validate_polygons and the
flag inside the IoU calls) against the exact rule of tests/validate_rule.py,
polygon by polygon, for K = 8 and K = 4 storage."""
import numpy as np
import pytest

from .gpu_helpers import dev, host
from .validate_rule import families, passes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dg():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2011_11134_gb300 as m

    m.dgal_get_device_status(clear=True)
    return m


def _expected(P, C):
    return np.array([0 if passes(p, int(m)) else 1 for p, m in zip(P, C)], np.uint8)


def test_validate_matches_exact_rule(dg):
    P, C, names = families(seed=9, n=400)
    want = _expected(P, C)
    assert 0 < want.sum() < len(want)
    dg.dgal_get_device_status(clear=True)
    bad = host(dg.dgal_validate_polygons(dev(P), dev(C)))
    wrong = np.nonzero(bad != want)[0]
    assert wrong.size == 0, [(names[i], P[i][: C[i]].tolist()) for i in wrong[:3]]
    assert dg.dgal_get_device_status(clear=True) & dg.DGAL_DEV_NOT_CONVEX
    # K = 4 storage: the polygons of at most 4 vertices
    q = np.nonzero(C <= 4)[0]
    P4, C4 = np.ascontiguousarray(P[q, :4]), C[q]
    bad4 = host(dg.dgal_validate_polygons(dev(P4), dev(C4)))
    assert (bad4 == want[q]).all()
    dg.dgal_get_device_status(clear=True)
    # only valid polygons: the status bit stays clear
    ok = np.nonzero(want == 0)[0]
    assert not host(dg.dgal_validate_polygons(dev(P[ok]), dev(C[ok]))).any()
    assert dg.dgal_get_device_status(clear=True) == 0


def test_validate_flag_in_paired_call(dg):
    import torch

    P, C, names = families(seed=10, n=64)
    want = _expected(P, C)
    ok = np.nonzero(want == 0)[0]
    p1, c1 = dev(P[ok]), dev(C[ok])
    p2, c2 = dev(P[ok][::-1].copy()), dev(C[ok][::-1].copy())
    dg.dgal_get_device_status(clear=True)
    a = dg.dgal_iou_paired(p1, p2, c1, c2, flags=dg.DGAL_FP64_REFINE | dg.DGAL_VALIDATE)
    b = dg.dgal_iou_paired(p1, p2, c1, c2, flags=dg.DGAL_FP64_REFINE)
    torch.cuda.synchronize()
    assert dg.dgal_get_device_status(clear=True) == 0
    assert torch.equal(a[0], b[0]) and torch.equal(a[2], b[2])
    # one clockwise polygon among them: the flag reports it
    badp = P[ok].copy()
    m = int(C[ok][0])
    badp[0, :m] = badp[0, :m][::-1]
    dg.dgal_iou_paired(dev(badp), p2, c1, c2, flags=dg.DGAL_FP64_REFINE | dg.DGAL_VALIDATE)
    assert dg.dgal_get_device_status(clear=True) & dg.DGAL_DEV_NOT_CONVEX
