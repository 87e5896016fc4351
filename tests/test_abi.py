"""The C ABI library builds for sm_103a, loads, and exports every symbol the
header declares (no compute calls: these run without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def libdgal():
    from paper_2011_11134_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def _declared():
    src = open(os.path.join(ROOT, "include", "dgal.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dgal_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_calls():
    names = _declared()
    for n in ("dgal_iou_paired", "dgal_iou_pairwise", "dgal_iou_backward", "dgal_iou_pairwise_batched",
              "dgal_batched_workspace_bytes", "dgal_autotune", "dgal_last_error", "dgal_get_device_status"):
        assert n in names


def test_library_exports_every_declared_symbol(libdgal):
    for name in _declared():
        assert hasattr(libdgal, name), name


def test_binding_covers_header():
    from paper_2011_11134_gb300 import _lib

    assert sorted(_lib.exported_symbols()) == _declared()


def test_host_only_calls(libdgal):
    libdgal.dgal_version.restype = ctypes.c_int
    assert libdgal.dgal_version() == 100
    libdgal.dgal_batched_workspace_bytes.restype = ctypes.c_size_t
    libdgal.dgal_batched_workspace_bytes.argtypes = [ctypes.c_int, ctypes.c_int]
    assert libdgal.dgal_batched_workspace_bytes(64, 4) >= 16 + 65 * 8
    assert libdgal.dgal_batched_workspace_bytes(64, 4) % 16 == 0


def test_validation_rejects_before_any_launch(libdgal):
    """Argument errors are caught on the host, so they are testable without a GPU."""
    f = libdgal.dgal_iou_paired
    P = ctypes.c_void_p
    f.argtypes = [P, P, P, P, ctypes.c_int64, ctypes.c_int, P, P, P, P, ctypes.c_uint32, P]
    f.restype = ctypes.c_int
    libdgal.dgal_last_error.restype = ctypes.c_char_p
    buf = (ctypes.c_float * 64)()
    base = ctypes.addressof(buf)
    al = base + (-base % 16)
    assert f(al, None, al, None, 4, 5, al, None, None, None, 0, None) == 2  # K unsupported
    assert f(al, None, al, None, -1, 4, al, None, None, None, 0, None) == 1  # negative n
    assert f(al, None, al, None, 0, 4, al, None, None, None, 0, None) == 0  # n = 0: no launch
    assert f(al + 4, None, al, None, 1, 4, al, None, None, None, 0, None) == 3  # misaligned polygons
    assert f(al, None, al, None, 1, 4, None, None, None, None, 0, None) == 1  # iou NULL
    assert f(al, None, al, None, 1, 4, al, al, None, None, 0, None) == 1  # nx without xflags
    assert b"xflags" in libdgal.dgal_last_error()


def test_nms_host_checks(libdgal):
    """NMS workspace sizing and its limits are host-side."""
    ws = libdgal.dgal_nms_workspace_bytes
    ws.restype = ctypes.c_size_t
    ws.argtypes = [ctypes.c_int64, ctypes.c_int]
    n = 1000
    words = (n + 63) // 64
    assert ws(n, 4) >= n * 4 + n * 32 + n + n * words * 8
    assert ws(n, 8) > ws(n, 4)
    assert ws(131072, 4) > 0 and ws(131073, 4) == 0 and ws(10, 5) == 0 and ws(-1, 4) == 0
    f = libdgal.dgal_nms_rotated
    P = ctypes.c_void_p
    f.argtypes = [P, P, P, ctypes.c_int64, ctypes.c_int, ctypes.c_float, P, P, P, ctypes.c_size_t, ctypes.c_uint32, P]
    f.restype = ctypes.c_int
    buf = (ctypes.c_double * 64)()
    base = ctypes.addressof(buf)
    al = base + (-base % 16)
    assert f(al, None, al, 10, 6, 0.5, al, al, al, 1 << 20, 0, None) == 2  # K unsupported
    assert f(al, None, al, 200000, 4, 0.5, al, al, al, 1 << 20, 0, None) == 1  # beyond the box limit
    assert f(al, None, al, 10, 4, 0.5, al, None, al, 1 << 20, 0, None) == 1  # num_keep NULL
    assert f(al, None, al, 10, 4, 0.5, al, al + 4, al, 1 << 20, 0, None) == 3  # num_keep misaligned
    assert f(al + 8, None, al, 10, 4, 0.5, al, al, al, 1 << 20, 0, None) == 3  # boxes misaligned
    assert f(al, None, al, 10, 4, 0.5, al, al, al, 16, 0, None) == 5  # workspace too small
    assert f(al, None, al, 10, 4, 0.5, al, al, None, 1 << 20, 0, None) == 5  # workspace NULL


def test_host_call_checks(libdgal):
    """dgal_iou_fwd_bwd_host validates its arguments on the host, before any
    device work; its workspace sizing is host arithmetic."""
    wsb = libdgal.dgal_iou_host_workspace_bytes
    wsb.restype = ctypes.c_size_t
    wsb.argtypes = [ctypes.c_int64, ctypes.c_int]
    assert wsb(1000, 4) >= 3 * 1000 * (2 * 32 + 4 + 4 + 1 + 8 + 2 * 32 + 2)
    assert wsb(1000, 8) > wsb(1000, 4) and wsb(1000, 5) == 0 and wsb(0, 4) == 0
    f = libdgal.dgal_iou_fwd_bwd_host
    P = ctypes.c_void_p
    f.argtypes = [P, P, P, P, P, ctypes.c_int64, ctypes.c_int, P, P, P, P, ctypes.c_size_t, ctypes.c_int64,
                  ctypes.c_uint32, P]
    f.restype = ctypes.c_int
    buf = (ctypes.c_float * 64)()
    a = ctypes.addressof(buf)
    assert f(a, None, a, None, a, 4, 5, a, a, a, None, 0, 16, 0, None) == 2  # K unsupported
    assert f(a, None, a, None, a, -1, 4, a, a, a, None, 0, 16, 0, None) == 1  # negative n
    assert f(a, None, a, None, a, 0, 4, a, a, a, None, 0, 16, 0, None) == 0  # n = 0: nothing to do
    assert f(a, None, a, None, a, 4, 4, a, a, a, None, 0, 0, 0, None) == 1  # chunk not positive
    assert f(a, None, a, None, None, 4, 4, a, a, a, None, 0, 16, 0, None) == 1  # grad NULL
    # pageable buffers take the staged form, which needs a workspace
    assert f(a, None, a, None, a, 4, 8, a, a, a, None, 0, 16, 0, None) == 5


def test_workspace_sizes_refuse_overflowing_counts(libdgal):
    """Sizing calls return 0 for pair counts whose workspace size would
    overflow (no such input fits in memory)."""
    for name in ("dgal_iou_host_workspace_bytes", "dgal_iou_loss_workspace_bytes"):
        f = getattr(libdgal, name)
        f.restype = ctypes.c_size_t
        f.argtypes = [ctypes.c_int64, ctypes.c_int]
        assert f(1 << 62, 4) == 0 and f(-5, 4) == 0


def test_noalloc_host_checks(libdgal):
    """The allocation-free ragged batch checks its arguments before its scene
    limit, and a call that succeeds clears the previous call's message."""
    f = libdgal.dgal_iou_pairwise_batched_noalloc
    P = ctypes.c_void_p
    f.argtypes = [ctypes.c_int, P, P, P, P, P, P, P, ctypes.c_int, P, P, ctypes.c_uint32, P]
    f.restype = ctypes.c_int
    libdgal.dgal_last_error.restype = ctypes.c_char_p
    buf = (ctypes.c_double * 64)()
    base = ctypes.addressof(buf)
    al = base + (-base % 16)
    assert f(5000, al, al, al, al, None, al, None, 5, al, None, 0, None) == 2  # K before the limit
    assert f(5000, None, al, al, al, None, al, None, 4, al, None, 0, None) == 1  # NULL offsets before the limit
    assert f(5000, al, al, al, al + 4, None, al, None, 4, al, None, 0, None) == 3  # misaligned polygons
    assert f(5000, al, al, al, al, None, al, None, 4, al, None, 0, None) == 5  # beyond 4096 scenes
    assert b"4096" in libdgal.dgal_last_error()
    assert f(0, None, None, None, None, None, None, None, 4, None, None, 0, None) == 0  # S = 0: no launch
    assert libdgal.dgal_last_error() == b""
