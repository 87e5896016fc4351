"""The allocation-free ragged batch, called through the C ABI.

Some callers cannot allocate device memory when they call the library (code
running during CUDA-graph capture, latency-critical loops where cudaMalloc
would stall the device, plugins whose framework owns every allocation).
dgal_iou_pairwise_batched_noalloc serves them with a fixed scratch array
inside the library.  This test checks that it returns the same IoU and nx as
dgal_iou_pairwise_batched with a caller workspace, on two calls in a row (the
second call must not depend on what the first left in the shared array).
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_2011_11134_gb300 import workloads as W

from .gpu_helpers import IOU_ATOL

pytestmark = pytest.mark.gpu


def test_noalloc_matches_workspace_form_twice():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2011_11134_gb300 import _lib

    lib = _lib.lib()
    P = ctypes.c_void_p
    fn = lib.dgal_iou_pairwise_batched_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_int, P, P, P, P, P, P, P, ctypes.c_int, P, P, ctypes.c_uint32, P]
    ref_fn = lib.dgal_iou_pairwise_batched

    for call, seed in enumerate((11, 12)):
        d = W.ragged_scenes_64(seed=seed, S=48, n_range=(1, 400), m_range=(1, 60))
        dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
        a, b = dev(d["a"]), dev(d["b"])
        ao, bo, oo = dev(d["a_off"]), dev(d["b_off"]), dev(d["out_off"])
        total = int(d["out_off"][-1])
        S = len(d["N"])
        iou = torch.full((total,), -1.0, device="cuda")
        nx = torch.full((total,), 0xEE, dtype=torch.uint8, device="cuda")
        ref_iou = torch.empty(total, device="cuda")
        ref_nx = torch.empty(total, dtype=torch.uint8, device="cuda")
        ws = torch.empty(lib.dgal_batched_workspace_bytes(S, 4), dtype=torch.uint8, device="cuda")
        s = _lib.stream_ptr()
        assert ref_fn(S, _lib.ptr(ao), _lib.ptr(bo), _lib.ptr(oo), _lib.ptr(a), None, _lib.ptr(b), None, 4,
                      _lib.ptr(ref_iou), _lib.ptr(ref_nx), _lib.ptr(ws), ws.numel(), _lib.DGAL_FP64_REFINE, s) == 0
        st = fn(S, _lib.ptr(ao), _lib.ptr(bo), _lib.ptr(oo), _lib.ptr(a), None, _lib.ptr(b), None, 4, _lib.ptr(iou),
                _lib.ptr(nx), _lib.DGAL_FP64_REFINE, s)
        assert st == 0, lib.dgal_last_error()
        torch.cuda.synchronize()
        err = (iou - ref_iou).abs().max().item()
        assert err <= IOU_ATOL, f"call {call}: max |dIoU| {err}"
        assert torch.equal(nx, ref_nx), f"call {call}: nx differs"

    # the largest batch the fixed scratch holds (4096 scenes, most of them
    # empty), which pins the scratch size arithmetic
    d = W.ragged_scenes_64(seed=13, S=4096, n_range=(0, 3), m_range=(0, 2))
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()
    a, b = dev(d["a"]), dev(d["b"])
    ao, bo, oo = dev(d["a_off"]), dev(d["b_off"]), dev(d["out_off"])
    total = int(d["out_off"][-1])
    assert len(d["N"]) == 4096 and total > 0
    iou = torch.full((total,), -1.0, device="cuda")
    nx = torch.full((total,), 0xEE, dtype=torch.uint8, device="cuda")
    ref_iou = torch.empty(total, device="cuda")
    ref_nx = torch.empty(total, dtype=torch.uint8, device="cuda")
    ws = torch.empty(lib.dgal_batched_workspace_bytes(4096, 4), dtype=torch.uint8, device="cuda")
    s = _lib.stream_ptr()
    assert ref_fn(4096, _lib.ptr(ao), _lib.ptr(bo), _lib.ptr(oo), _lib.ptr(a), None, _lib.ptr(b), None, 4,
                  _lib.ptr(ref_iou), _lib.ptr(ref_nx), _lib.ptr(ws), ws.numel(), _lib.DGAL_FP64_REFINE, s) == 0
    st = fn(4096, _lib.ptr(ao), _lib.ptr(bo), _lib.ptr(oo), _lib.ptr(a), None, _lib.ptr(b), None, 4, _lib.ptr(iou),
            _lib.ptr(nx), _lib.DGAL_FP64_REFINE, s)
    assert st == 0, lib.dgal_last_error()
    torch.cuda.synchronize()
    assert (iou - ref_iou).abs().max().item() <= IOU_ATOL
    assert torch.equal(nx, ref_nx)

    # more scenes than the fixed scratch holds: a clear error, no launch
    big = torch.zeros(4098, dtype=torch.int64, device="cuda")
    st = fn(4097, _lib.ptr(big), _lib.ptr(big), _lib.ptr(big), _lib.ptr(a), None, _lib.ptr(b), None, 4,
            _lib.ptr(iou), _lib.ptr(nx), 0, _lib.stream_ptr())
    assert st == 5  # DGAL_ERR_WORKSPACE
    assert b"4096" in lib.dgal_last_error()
