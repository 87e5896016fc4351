"""ctypes binding of libdgal (include/dgal.h): argument marshalling only.

Every computation runs in the library's CUDA kernels.  PyTorch supplies
device memory and the current stream.  If the library has not been built,
every call raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdgal.so")

DGAL_OK = 0
DGAL_FP64_REFINE = 0x1
DGAL_PLAIN = 0x2
DGAL_LOSS_GIOU = 0x4
DGAL_LOSS_DIOU = 0x8
DGAL_VALIDATE = 0x10
DGAL_TEST_EXPIRE_WAIT = 0x100
DGAL_DEV_TIMEOUT = 0x10
DGAL_DEV_BAD_COUNT = 0x1
DGAL_DEV_OVERFLOW = 0x2
DGAL_DEV_BAD_FLAGS = 0x4
DGAL_DEV_BAD_OFFSETS = 0x8
DGAL_DEV_NOT_CONVEX = 0x20

STATUS_NAMES = {0: "DGAL_OK", 1: "DGAL_ERR_INVALID_ARG", 2: "DGAL_ERR_UNSUPPORTED_K", 3: "DGAL_ERR_ALIGNMENT",
                4: "DGAL_ERR_CUDA", 5: "DGAL_ERR_WORKSPACE", 6: "DGAL_ERR_DEVICE_STATUS"}

# name -> (restype, argtypes)
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_I = ctypes.c_int
_U32 = ctypes.c_uint32
_SIG = {
    "dgal_iou_paired": (_I, [_P, _P, _P, _P, _I64, _I, _P, _P, _P, _P, _U32, _P]),
    "dgal_iou_backward": (_I, [_P, _P, _P, _P, _I64, _I, _P, _P, _P, _P, _P, _U32, _P]),
    "dgal_iou_fwd_bwd": (_I, [_P, _P, _P, _P, _P, _I64, _I, _P, _P, _P, _P, _P, _U32, _P]),
    "dgal_iou_pairwise": (_I, [_P, _P, _I64, _P, _P, _I64, _I, _P, _P, _U32, _P]),
    "dgal_iou_loss_workspace_bytes": (ctypes.c_size_t, [_I64, _I]),
    "dgal_iou_loss": (_I, [_P, _P, _P, _P, _I64, _I, _P, ctypes.c_float, _P, _P, _P, _P, _P, ctypes.c_size_t, _U32, _P]),
    "dgal_iou_loss_backward": (_I, [_P, _P, _P, _P, _I64, _I, _P, ctypes.c_float, _P, _P, _P, _P, ctypes.c_size_t,
                                     _U32, _P]),
    "dgal_iou3d_loss_backward": (_I, [_P, _P, _P, _P, _P, _P, _I64, _I, _P, ctypes.c_float, _P, _P, _P, _P, _P, _P,
                                       ctypes.c_size_t, _U32, _P]),
    "dgal_iou3d_paired": (_I, [_P, _P, _P, _P, _P, _P, _I64, _I, _P, _P, _P, _P, _U32, _P]),
    "dgal_iou3d_backward": (_I, [_P, _P, _P, _P, _P, _P, _I64, _I, _P, _P, _P, _P, _P, _P, _P, _U32, _P]),
    "dgal_iou3d_loss": (_I, [_P, _P, _P, _P, _P, _P, _I64, _I, _P, ctypes.c_float, _P, _P, _P, _P, _P, _P, _P,
                             ctypes.c_size_t, _U32, _P]),
    "dgal_batched_workspace_bytes": (ctypes.c_size_t, [_I, _I]),
    "dgal_iou_pairwise_batched": (_I, [_I, _P, _P, _P, _P, _P, _P, _P, _I, _P, _P, _P, ctypes.c_size_t, _U32, _P]),
    "dgal_iou_pairwise_per_scene": (_I, [_I, _P, _P, _P, _P, _P, _P, _P, _I, _P, _P, _U32, _P]),
    "dgal_iou_pairwise_batched_noalloc": (_I, [_I, _P, _P, _P, _P, _P, _P, _P, _I, _P, _P, _U32, _P]),
    "dgal_batched_graph_create": (_I, [ctypes.POINTER(_P), _I, _P, _P, _P, _P, _P, _P, _P, _I, _P, _P, _P,
                                       ctypes.c_size_t, _U32]),
    "dgal_nms_workspace_bytes": (ctypes.c_size_t, [_I64, _I]),
    "dgal_nms_rotated": (_I, [_P, _P, _P, _I64, _I, ctypes.c_float, _P, _P, _P, ctypes.c_size_t, _U32, _P]),
    "dgal_intersect_paired": (_I, [_P, _P, _P, _P, _I64, _I, _P, _P, _P, _P, _U32, _P]),
    "dgal_area": (_I, [_P, _P, _I64, _I, _P, _P]),
    "dgal_validate_polygons": (_I, [_P, _P, _I64, _I, _P, _P]),
    "dgal_line_from_points": (_I, [_P, _P, _I64, _P, _P]),
    "dgal_line_from_points_backward": (_I, [_P, _P, _I64, _P, _P, _P, _P]),
    "dgal_line_intersect": (_I, [_P, _P, _I64, _P, _P]),
    "dgal_line_intersect_backward": (_I, [_P, _P, _I64, _P, _P, _P, _P]),
    "dgal_iou_host_workspace_bytes": (ctypes.c_size_t, [_I64, _I]),
    "dgal_iou_fwd_bwd_host": (_I, [_P, _P, _P, _P, _P, _I64, _I, _P, _P, _P, _P, ctypes.c_size_t, _I64, _U32, _P]),
    "dgal_graph_launch": (_I, [_P, _P]),
    "dgal_graph_destroy": (_I, [_P]),
    "dgal_autotune": (_I, [_I, _I, ctypes.c_char_p]),
    "dgal_get_batched_config": (_I, [_I, ctypes.POINTER(ctypes.c_int32)]),
    "dgal_get_paired_config": (_I, [_I, ctypes.POINTER(ctypes.c_int64)]),
    "dgal_get_device_status": (_I, [ctypes.POINTER(_U32), _I]),
    "dgal_last_error": (ctypes.c_char_p, []),
    "dgal_version": (_I, []),
}

_lock = threading.Lock()
_lib = None


class DgalError(RuntimeError):
    def __init__(self, call: str, status: int, msg: str):
        super().__init__(f"{call} failed: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def lib():
    """The loaded libdgal (raises if it has not been built)."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise RuntimeError(
                        f"libdgal.so is not built ({LIB_PATH} missing): run "
                        "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc); "
                        "there is no CPU fallback")
                L = ctypes.CDLL(LIB_PATH)
                for name, (res, args) in _SIG.items():
                    fn = getattr(L, name)
                    fn.restype = res
                    fn.argtypes = args
                _lib = L
    return _lib


def exported_symbols():
    return list(_SIG)


def call(name: str, *args):
    st = getattr(lib(), name)(*args)
    if st != DGAL_OK:
        msg = lib().dgal_last_error().decode(errors="replace")
        raise DgalError(name, st, msg)
    return st


def ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)
