"""GB300 (sm_103a) convex-polygon IoU with a hand-written backward (DGAL, arXiv:2011.11134).

Python binding of libdgal's C ABI (include/dgal.h), with the same call names:

    dgal_iou_paired            paper Sec. II-B `iou`: IoU, nx, xflags per pair
    dgal_iou_backward          paper Sec. II-B `iou_backward`: dL/dIoU -> vertex grads
    dgal_iou_pairwise          N x M IoU matrix
    dgal_iou_pairwise_batched  ragged scenes in one persistent launch
    dgal_iou_pairwise_per_scene  the plain one-launch-per-scene form
    dgal_nms_rotated           greedy rotated NMS on the pairwise IoU
    dgal_intersect_paired      paper Sec. II-B `intersect`: the intersection polygon
    dgal_area                  paper Sec. II-B `area` of single polygons
    dgal_line_*                paper Sec. III lines: from two points, intersection (+ backward)
    BatchedGraph               the ragged batch captured in a CUDA graph
    dgal_autotune              launch-shape tuner for the ragged batch
    dgal_get_device_status     device-side error bits
    dgal_validate_polygons     input check: strictly convex, counter-clockwise
                               (also run inside a call by flags=DGAL_VALIDATE)

and ``IoU`` / ``iou``: a ``torch.autograd.Function`` whose backward consumes
the recorded (nx, xflags) or, in recompute mode, re-runs the clip.

Polygons are float32 CUDA tensors [n, K, 2] (K = 4 or 8, counter-clockwise,
convex) with optional uint8 vertex counts [n].  Everything runs in the
library's kernels on the current CUDA stream; this module only checks and
marshals arguments.  ``workloads`` (seeded inputs) imports without CUDA.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import _lib
from ._lib import (DGAL_DEV_BAD_COUNT, DGAL_DEV_BAD_FLAGS, DGAL_DEV_BAD_OFFSETS, DGAL_DEV_OVERFLOW,
                   DGAL_DEV_NOT_CONVEX, DGAL_DEV_TIMEOUT, DGAL_FP64_REFINE, DGAL_LOSS_DIOU, DGAL_LOSS_GIOU,
                   DGAL_PLAIN, DGAL_TEST_EXPIRE_WAIT, DGAL_VALIDATE, DgalError)

__all__ = [
    "dgal_iou_paired", "dgal_iou_backward", "dgal_iou_fwd_bwd", "dgal_iou_pairwise", "dgal_iou_pairwise_batched",
    "dgal_iou_pairwise_per_scene", "dgal_batched_workspace_bytes", "BatchedGraph", "dgal_autotune",
    "dgal_iou_loss", "dgal_iou_loss_workspace_bytes", "dgal_iou_loss_backward", "dgal_iou3d_loss_backward",
    "IoULoss", "iou_loss", "DGAL_LOSS_GIOU", "DGAL_LOSS_DIOU", "LOSS_VARIANTS", "DGAL_DEV_TIMEOUT",
    "DGAL_TEST_EXPIRE_WAIT",
    "dgal_get_batched_config", "dgal_get_paired_config", "dgal_get_device_status", "dgal_last_error", "dgal_version", "IoU", "iou",
    "DGAL_FP64_REFINE", "DGAL_PLAIN", "DGAL_DEV_BAD_COUNT", "DGAL_DEV_OVERFLOW", "DGAL_DEV_BAD_FLAGS",
    "DGAL_DEV_BAD_OFFSETS", "DgalError", "dgal_iou3d_paired", "dgal_iou3d_backward", "dgal_iou3d_loss", "IoU3D",
    "iou3d", "IoU3DLoss", "iou3d_loss", "dgal_nms_rotated", "dgal_nms_workspace_bytes",
    "dgal_intersect_paired", "dgal_area", "dgal_line_from_points", "dgal_line_from_points_backward",
    "dgal_line_intersect", "dgal_line_intersect_backward", "LineFromPoints", "LineIntersect",
    "line_from_points", "line_intersect", "dgal_iou_fwd_bwd_host", "dgal_iou_host_workspace_bytes",
    "dgal_validate_polygons", "DGAL_VALIDATE", "DGAL_DEV_NOT_CONVEX",
]


def _poly(t, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float32 or t.dim() != 3 or t.shape[2] != 2 or t.shape[1] not in (4, 8):
        raise ValueError(f"{name} must be float32 [n, K, 2] with K in (4, 8), got {tuple(t.shape)} {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t


def _counts(c, n, name, device):
    if c is None:
        return None
    if not isinstance(c, torch.Tensor) or c.dtype != torch.uint8 or c.shape != (n,) or not c.is_contiguous():
        raise ValueError(f"{name} must be a contiguous uint8 tensor of shape ({n},)")
    if c.device != device:
        raise ValueError(f"{name} must be on {device}")
    return c


def dgal_iou_paired(p1, p2, c1=None, c2=None, save_flags=True, with_degen=False, flags=DGAL_FP64_REFINE,
                    stream=None):
    """IoU of paired polygons; returns (iou [n], nx [n] | None, xflags [n, 2K] | None, degen [n] | None)."""
    _poly(p1, "p1")
    _poly(p2, "p2")
    if p1.shape != p2.shape or p1.device != p2.device:
        raise ValueError("p1 and p2 must have the same shape and device")
    n, K = p1.shape[0], p1.shape[1]
    c1 = _counts(c1, n, "c1", p1.device)
    c2 = _counts(c2, n, "c2", p1.device)
    iou = torch.empty(n, device=p1.device, dtype=torch.float32)
    nx = torch.empty(n, device=p1.device, dtype=torch.uint8) if save_flags else None
    xflags = torch.empty((n, 2 * K), device=p1.device, dtype=torch.uint8) if save_flags else None
    degen = torch.empty(n, device=p1.device, dtype=torch.uint8) if with_degen else None
    _lib.call("dgal_iou_paired", _lib.ptr(p1), _lib.ptr(c1), _lib.ptr(p2), _lib.ptr(c2), n, K, _lib.ptr(iou),
              _lib.ptr(nx), _lib.ptr(xflags), _lib.ptr(degen), flags, _lib.stream_ptr(stream))
    return iou, nx, xflags, degen


def dgal_iou_backward(p1, p2, grad_iou, nx=None, xflags=None, c1=None, c2=None, flags=DGAL_FP64_REFINE,
                      stream=None):
    """dL/dIoU [n] -> (dL/dp1, dL/dp2), each [n, K, 2].  nx/xflags None -> recompute the clip."""
    _poly(p1, "p1")
    _poly(p2, "p2")
    n, K = p1.shape[0], p1.shape[1]
    if grad_iou.dtype != torch.float32 or grad_iou.shape != (n,) or not grad_iou.is_cuda:
        raise ValueError("grad_iou must be a CUDA float32 tensor of shape (n,)")
    grad_iou = grad_iou.contiguous()
    c1 = _counts(c1, n, "c1", p1.device)
    c2 = _counts(c2, n, "c2", p1.device)
    if (nx is None) != (xflags is None):
        raise ValueError("nx and xflags must be given together")
    if nx is not None and (nx.shape != (n,) or xflags.shape != (n, 2 * K)):
        raise ValueError("nx must be [n] and xflags [n, 2K]")
    g1 = torch.empty_like(p1)
    g2 = torch.empty_like(p2)
    _lib.call("dgal_iou_backward", _lib.ptr(p1), _lib.ptr(c1), _lib.ptr(p2), _lib.ptr(c2), n, K,
              _lib.ptr(grad_iou), _lib.ptr(nx), _lib.ptr(xflags), _lib.ptr(g1), _lib.ptr(g2), flags,
              _lib.stream_ptr(stream))
    return g1, g2


def dgal_iou_fwd_bwd(p1, p2, grad_iou, c1=None, c2=None, flags=DGAL_FP64_REFINE, stream=None):
    """Forward and backward in one call when dL/dIoU is known up front:
    returns (iou [n], dL/dp1, dL/dp2 [n, K, 2]).  K = 4 runs one kernel (no
    flags are stored); K = 8 saves the flags in scratch this call allocates."""
    _poly(p1, "p1")
    _poly(p2, "p2")
    n, K = p1.shape[0], p1.shape[1]
    if grad_iou.dtype != torch.float32 or grad_iou.shape != (n,) or not grad_iou.is_cuda:
        raise ValueError("grad_iou must be a CUDA float32 tensor of shape (n,)")
    grad_iou = grad_iou.contiguous()
    c1 = _counts(c1, n, "c1", p1.device)
    c2 = _counts(c2, n, "c2", p1.device)
    iou = torch.empty(n, device=p1.device, dtype=torch.float32)
    g1 = torch.empty_like(p1)
    g2 = torch.empty_like(p2)
    nx = xf = None
    if K != 4:
        nx = torch.empty(n, device=p1.device, dtype=torch.uint8)
        xf = torch.empty((n, 2 * K), device=p1.device, dtype=torch.uint8)
    _lib.call("dgal_iou_fwd_bwd", _lib.ptr(p1), _lib.ptr(c1), _lib.ptr(p2), _lib.ptr(c2), _lib.ptr(grad_iou), n, K,
              _lib.ptr(iou), _lib.ptr(g1), _lib.ptr(g2), _lib.ptr(nx), _lib.ptr(xf), flags, _lib.stream_ptr(stream))
    return iou, g1, g2


def dgal_iou_loss_workspace_bytes(n, K=4):
    return int(_lib.lib().dgal_iou_loss_workspace_bytes(n, K))


# loss variant name -> flag bits of dgal_iou_loss
LOSS_VARIANTS = {"iou": 0, "giou": DGAL_LOSS_GIOU, "diou": DGAL_LOSS_DIOU}


def _loss_flags(flags, variant):
    if variant not in LOSS_VARIANTS:
        raise ValueError(f"variant must be one of {sorted(LOSS_VARIANTS)}")
    return (flags & ~(DGAL_LOSS_GIOU | DGAL_LOSS_DIOU)) | LOSS_VARIANTS[variant]


def dgal_iou_loss(p1, p2, weight=None, scale=1.0, c1=None, c2=None, grads=True, with_iou=False,
                  flags=DGAL_FP64_REFINE, stream=None, workspace=None, out=None, variant="iou"):
    """IoU loss (K = 4 or 8): returns (loss [1], g1 | None, g2 | None, iou | None)
    with loss = scale * sum w (1 - IoU) (variant "iou"), scale * sum w (1 -
    GIoU) ("giou") or scale * sum w (1 - DIoU) ("diou"), and g = d loss / d p.
    `workspace` (uint8, dgal_iou_loss_workspace_bytes(n, K) bytes) holds the
    per-warp partials and the state passed from the forward to the backward;
    after a call with grads=False it feeds dgal_iou_loss_backward."""
    flags = _loss_flags(flags, variant)
    _poly(p1, "p1")
    _poly(p2, "p2")
    if p1.shape != p2.shape:
        raise ValueError("p1 and p2 must have the same shape")
    n, K = p1.shape[0], p1.shape[1]
    c1 = _counts(c1, n, "c1", p1.device)
    c2 = _counts(c2, n, "c2", p1.device)
    if weight is not None and (weight.dtype != torch.float32 or weight.shape != (n,) or not weight.is_contiguous()):
        raise ValueError("weight must be a contiguous float32 tensor of shape (n,)")
    if workspace is None:
        workspace = torch.empty(max(dgal_iou_loss_workspace_bytes(n, K), 16), device=p1.device, dtype=torch.uint8)
    if out is None:
        loss = torch.empty(1, device=p1.device, dtype=torch.float32)
        g1 = torch.empty_like(p1) if grads else None
        g2 = torch.empty_like(p2) if grads else None
        iou = torch.empty(n, device=p1.device, dtype=torch.float32) if with_iou else None
    else:
        loss, g1, g2, iou = out
    _lib.call("dgal_iou_loss", _lib.ptr(p1), _lib.ptr(c1), _lib.ptr(p2), _lib.ptr(c2), n, K, _lib.ptr(weight),
              float(scale), _lib.ptr(loss), _lib.ptr(iou), _lib.ptr(g1), _lib.ptr(g2), _lib.ptr(workspace),
              workspace.numel(), flags, _lib.stream_ptr(stream))
    return loss, g1, g2, iou


def dgal_iou_loss_backward(p1, p2, workspace, dloss=None, weight=None, scale=1.0, c1=None, c2=None,
                           flags=DGAL_FP64_REFINE, stream=None, variant="iou"):
    """Gradients of a loss computed by dgal_iou_loss(grads=False) with this
    workspace: returns (g1, g2) = dloss * d loss / d p1, d p2, with dloss a
    CUDA float32 tensor of one element (read on the device) or None (1)."""
    flags = _loss_flags(flags, variant)
    n, K = p1.shape[0], p1.shape[1]
    if dloss is not None and (not isinstance(dloss, torch.Tensor) or dloss.dtype != torch.float32 or
                              dloss.numel() != 1 or dloss.device != p1.device):
        raise ValueError("dloss must be a float32 tensor of one element on the polygons' device")
    dloss = None if dloss is None else dloss.contiguous()
    g1, g2 = torch.empty_like(p1), torch.empty_like(p2)
    _lib.call("dgal_iou_loss_backward", _lib.ptr(p1), _lib.ptr(c1), _lib.ptr(p2), _lib.ptr(c2), n, K, _lib.ptr(weight),
              float(scale), _lib.ptr(dloss), _lib.ptr(g1), _lib.ptr(g2), _lib.ptr(workspace), workspace.numel(), flags,
              _lib.stream_ptr(stream))
    return g1, g2


def dgal_iou3d_loss_backward(p1, z1, p2, z2, workspace, dloss=None, weight=None, scale=1.0, c1=None, c2=None,
                             flags=DGAL_FP64_REFINE, stream=None):
    """Gradients of a loss computed by dgal_iou3d_loss(grads=False) with this
    workspace: returns (g1, gz1, g2, gz2), each times dloss (see
    dgal_iou_loss_backward)."""
    n, K = p1.shape[0], p1.shape[1]
    if dloss is not None and (not isinstance(dloss, torch.Tensor) or dloss.dtype != torch.float32 or
                              dloss.numel() != 1 or dloss.device != p1.device):
        raise ValueError("dloss must be a float32 tensor of one element on the polygons' device")
    dloss = None if dloss is None else dloss.contiguous()
    g1, g2, gz1, gz2 = torch.empty_like(p1), torch.empty_like(p2), torch.empty_like(z1), torch.empty_like(z2)
    _lib.call("dgal_iou3d_loss_backward", _lib.ptr(p1), _lib.ptr(c1), _lib.ptr(z1), _lib.ptr(p2), _lib.ptr(c2),
              _lib.ptr(z2), n, K, _lib.ptr(weight), float(scale), _lib.ptr(dloss), _lib.ptr(g1), _lib.ptr(gz1),
              _lib.ptr(g2), _lib.ptr(gz2), _lib.ptr(workspace), workspace.numel(), flags, _lib.stream_ptr(stream))
    return g1, gz1, g2, gz2


def _zext(z, n, name, device):
    if not isinstance(z, torch.Tensor) or z.dtype != torch.float32 or z.shape != (n, 2) or not z.is_contiguous():
        raise ValueError(f"{name} must be a contiguous float32 tensor of shape ({n}, 2) = (z_center, height)")
    if z.device != device:
        raise ValueError(f"{name} must be on {device}")
    return z


def dgal_iou3d_paired(p1, z1, p2, z2, c1=None, c2=None, save_flags=True, with_degen=False, flags=DGAL_FP64_REFINE,
                      stream=None):
    """3D IoU of paired boxes (bird's-eye-view polygon [n, K, 2] + vertical
    extent [n, 2] = (z_center, height)); returns (iou [n], nx | None,
    xflags | None, degen | None) with the bird's-eye-view flags."""
    _poly(p1, "p1")
    _poly(p2, "p2")
    if p1.shape != p2.shape or p1.device != p2.device:
        raise ValueError("p1 and p2 must have the same shape and device")
    n, K = p1.shape[0], p1.shape[1]
    z1, z2 = _zext(z1, n, "z1", p1.device), _zext(z2, n, "z2", p1.device)
    c1 = _counts(c1, n, "c1", p1.device)
    c2 = _counts(c2, n, "c2", p1.device)
    iou = torch.empty(n, device=p1.device, dtype=torch.float32)
    nx = torch.empty(n, device=p1.device, dtype=torch.uint8) if save_flags else None
    xflags = torch.empty((n, 2 * K), device=p1.device, dtype=torch.uint8) if save_flags else None
    degen = torch.empty(n, device=p1.device, dtype=torch.uint8) if with_degen else None
    _lib.call("dgal_iou3d_paired", _lib.ptr(p1), _lib.ptr(c1), _lib.ptr(z1), _lib.ptr(p2), _lib.ptr(c2), _lib.ptr(z2),
              n, K, _lib.ptr(iou), _lib.ptr(nx), _lib.ptr(xflags), _lib.ptr(degen), flags, _lib.stream_ptr(stream))
    return iou, nx, xflags, degen


def dgal_iou3d_backward(p1, z1, p2, z2, grad_iou, nx=None, xflags=None, c1=None, c2=None, flags=DGAL_FP64_REFINE,
                        stream=None):
    """dL/dIoU3 [n] -> (dL/dp1 [n,K,2], dL/dz1 [n,2], dL/dp2, dL/dz2)."""
    _poly(p1, "p1")
    _poly(p2, "p2")
    n, K = p1.shape[0], p1.shape[1]
    z1, z2 = _zext(z1, n, "z1", p1.device), _zext(z2, n, "z2", p1.device)
    if grad_iou.dtype != torch.float32 or grad_iou.shape != (n,) or not grad_iou.is_cuda:
        raise ValueError("grad_iou must be a CUDA float32 tensor of shape (n,)")
    grad_iou = grad_iou.contiguous()
    c1 = _counts(c1, n, "c1", p1.device)
    c2 = _counts(c2, n, "c2", p1.device)
    if (nx is None) != (xflags is None):
        raise ValueError("nx and xflags must be given together")
    g1, g2 = torch.empty_like(p1), torch.empty_like(p2)
    gz1, gz2 = torch.empty_like(z1), torch.empty_like(z2)
    _lib.call("dgal_iou3d_backward", _lib.ptr(p1), _lib.ptr(c1), _lib.ptr(z1), _lib.ptr(p2), _lib.ptr(c2),
              _lib.ptr(z2), n, K, _lib.ptr(grad_iou), _lib.ptr(nx), _lib.ptr(xflags), _lib.ptr(g1), _lib.ptr(gz1),
              _lib.ptr(g2), _lib.ptr(gz2), flags, _lib.stream_ptr(stream))
    return g1, gz1, g2, gz2


def dgal_iou3d_loss(p1, z1, p2, z2, weight=None, scale=1.0, c1=None, c2=None, grads=True, with_iou=False,
                    flags=DGAL_FP64_REFINE, stream=None, workspace=None):
    """3D IoU loss: returns (loss [1], g1, gz1, g2, gz2, iou) (gradients None
    when grads is False) with loss = scale * sum w (1 - IoU3)."""
    _poly(p1, "p1")
    _poly(p2, "p2")
    if p1.shape != p2.shape:
        raise ValueError("p1 and p2 must have the same shape")
    n, K = p1.shape[0], p1.shape[1]
    z1, z2 = _zext(z1, n, "z1", p1.device), _zext(z2, n, "z2", p1.device)
    c1 = _counts(c1, n, "c1", p1.device)
    c2 = _counts(c2, n, "c2", p1.device)
    if weight is not None and (weight.dtype != torch.float32 or weight.shape != (n,) or not weight.is_contiguous()):
        raise ValueError("weight must be a contiguous float32 tensor of shape (n,)")
    if workspace is None:
        workspace = torch.empty(max(dgal_iou_loss_workspace_bytes(n, K), 16), device=p1.device, dtype=torch.uint8)
    loss = torch.empty(1, device=p1.device, dtype=torch.float32)
    g1 = torch.empty_like(p1) if grads else None
    g2 = torch.empty_like(p2) if grads else None
    gz1 = torch.empty_like(z1) if grads else None
    gz2 = torch.empty_like(z2) if grads else None
    iou = torch.empty(n, device=p1.device, dtype=torch.float32) if with_iou else None
    _lib.call("dgal_iou3d_loss", _lib.ptr(p1), _lib.ptr(c1), _lib.ptr(z1), _lib.ptr(p2), _lib.ptr(c2), _lib.ptr(z2),
              n, K, _lib.ptr(weight), float(scale), _lib.ptr(loss), _lib.ptr(iou), _lib.ptr(g1), _lib.ptr(gz1),
              _lib.ptr(g2), _lib.ptr(gz2), _lib.ptr(workspace), workspace.numel(), flags, _lib.stream_ptr(stream))
    return loss, g1, gz1, g2, gz2, iou


def dgal_iou_pairwise(a, b, ca=None, cb=None, with_nx=True, flags=DGAL_FP64_REFINE, stream=None, out=None):
    """N x M IoU matrix; returns (iou [N, M], nx [N, M] | None)."""
    _poly(a, "a")
    _poly(b, "b")
    N, M, K = a.shape[0], b.shape[0], a.shape[1]
    if b.shape[1] != K:
        raise ValueError("a and b must have the same K")
    ca = _counts(ca, N, "ca", a.device)
    cb = _counts(cb, M, "cb", a.device)
    if out is None:
        iou = torch.empty((N, M), device=a.device, dtype=torch.float32)
        nx = torch.empty((N, M), device=a.device, dtype=torch.uint8) if with_nx else None
    else:
        iou, nx = out
    _lib.call("dgal_iou_pairwise", _lib.ptr(a), _lib.ptr(ca), N, _lib.ptr(b), _lib.ptr(cb), M, K, _lib.ptr(iou),
              _lib.ptr(nx), flags, _lib.stream_ptr(stream))
    return iou, nx


def dgal_intersect_paired(p1, p2, c1=None, c2=None, flags=DGAL_FP64_REFINE, stream=None):
    """The intersection polygon of each pair (paper Sec. II-B `intersect`):
    returns (verts [n, 2K, 2] in xflags order, unused slots 0, area [n],
    nx [n], xflags [n, 2K])."""
    _poly(p1, "p1")
    _poly(p2, "p2")
    if p1.shape != p2.shape or p1.device != p2.device:
        raise ValueError("p1 and p2 must have the same shape and device")
    n, K = p1.shape[0], p1.shape[1]
    c1 = _counts(c1, n, "c1", p1.device)
    c2 = _counts(c2, n, "c2", p1.device)
    verts = torch.empty((n, 2 * K, 2), device=p1.device, dtype=torch.float32)
    area = torch.empty(n, device=p1.device, dtype=torch.float32)
    nx = torch.empty(n, device=p1.device, dtype=torch.uint8)
    xflags = torch.empty((n, 2 * K), device=p1.device, dtype=torch.uint8)
    _lib.call("dgal_intersect_paired", _lib.ptr(p1), _lib.ptr(c1), _lib.ptr(p2), _lib.ptr(c2), n, K,
              _lib.ptr(verts), _lib.ptr(area), _lib.ptr(nx), _lib.ptr(xflags), flags, _lib.stream_ptr(stream))
    return verts, area, nx, xflags


def dgal_validate_polygons(p, c=None, stream=None):
    """Input check of polygons [n, K, 2] (with counts c): uint8 [n], 1 where a
    polygon is not strictly convex in counter-clockwise order (such a polygon
    also sets DGAL_DEV_NOT_CONVEX in the device status word)."""
    _poly(p, "p")
    n, K = p.shape[0], p.shape[1]
    c = _counts(c, n, "c", p.device)
    bad = torch.empty(n, device=p.device, dtype=torch.uint8)
    _lib.call("dgal_validate_polygons", _lib.ptr(p), _lib.ptr(c), n, K, _lib.ptr(bad), _lib.stream_ptr(stream))
    return bad


def dgal_area(p, c=None, stream=None):
    """Shoelace area of each polygon [n, K, 2] (paper Sec. II-B `area`)."""
    _poly(p, "p")
    n, K = p.shape[0], p.shape[1]
    c = _counts(c, n, "c", p.device)
    area = torch.empty(n, device=p.device, dtype=torch.float32)
    _lib.call("dgal_area", _lib.ptr(p), _lib.ptr(c), n, K, _lib.ptr(area), _lib.stream_ptr(stream))
    return area


def _pts(t, name, width):
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32 or t.dim() != 2 \
            or t.shape[1] != width or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA float32 tensor [n, {width}]")
    return t


def dgal_line_from_points(p, q, stream=None):
    """Lines through p[k], q[k] ([n, 2]): (a, b, c) [n, 3] with a x + b y + c = 0."""
    _pts(p, "p", 2)
    _pts(q, "q", 2)
    line = torch.empty((p.shape[0], 3), device=p.device, dtype=torch.float32)
    _lib.call("dgal_line_from_points", _lib.ptr(p), _lib.ptr(q), p.shape[0], _lib.ptr(line), _lib.stream_ptr(stream))
    return line


def dgal_line_from_points_backward(p, q, grad_line, stream=None):
    _pts(p, "p", 2)
    _pts(q, "q", 2)
    _pts(grad_line, "grad_line", 3)
    gp, gq = torch.empty_like(p), torch.empty_like(q)
    _lib.call("dgal_line_from_points_backward", _lib.ptr(p), _lib.ptr(q), p.shape[0], _lib.ptr(grad_line),
              _lib.ptr(gp), _lib.ptr(gq), _lib.stream_ptr(stream))
    return gp, gq


def dgal_line_intersect(l1, l2, stream=None):
    """Intersection points [n, 2] of lines l1[k], l2[k] ([n, 3] each)."""
    _pts(l1, "l1", 3)
    _pts(l2, "l2", 3)
    pt = torch.empty((l1.shape[0], 2), device=l1.device, dtype=torch.float32)
    _lib.call("dgal_line_intersect", _lib.ptr(l1), _lib.ptr(l2), l1.shape[0], _lib.ptr(pt), _lib.stream_ptr(stream))
    return pt


def dgal_line_intersect_backward(l1, l2, grad_point, stream=None):
    _pts(l1, "l1", 3)
    _pts(l2, "l2", 3)
    _pts(grad_point, "grad_point", 2)
    g1, g2 = torch.empty_like(l1), torch.empty_like(l2)
    _lib.call("dgal_line_intersect_backward", _lib.ptr(l1), _lib.ptr(l2), l1.shape[0], _lib.ptr(grad_point),
              _lib.ptr(g1), _lib.ptr(g2), _lib.stream_ptr(stream))
    return g1, g2


class LineFromPoints(torch.autograd.Function):
    """Differentiable line through two points (paper Sec. III, "Lines")."""

    @staticmethod
    def forward(ctx, p, q):
        p, q = p.contiguous(), q.contiguous()
        ctx.save_for_backward(p, q)
        return dgal_line_from_points(p, q)

    @staticmethod
    def backward(ctx, g):
        p, q = ctx.saved_tensors
        return dgal_line_from_points_backward(p, q, g.contiguous())


class LineIntersect(torch.autograd.Function):
    """Differentiable intersection point of two lines."""

    @staticmethod
    def forward(ctx, l1, l2):
        l1, l2 = l1.contiguous(), l2.contiguous()
        ctx.save_for_backward(l1, l2)
        return dgal_line_intersect(l1, l2)

    @staticmethod
    def backward(ctx, g):
        l1, l2 = ctx.saved_tensors
        return dgal_line_intersect_backward(l1, l2, g.contiguous())


def line_from_points(p, q):
    return LineFromPoints.apply(p, q)


def line_intersect(l1, l2):
    return LineIntersect.apply(l1, l2)


def dgal_iou_host_workspace_bytes(chunk, K=4):
    return int(_lib.lib().dgal_iou_host_workspace_bytes(chunk, K))


def dgal_iou_fwd_bwd_host(p1, p2, grad, c1=None, c2=None, out=None, chunk=131072, workspace=None,
                          flags=DGAL_FP64_REFINE, stream=None, device=None):
    """Paired IoU forward + backward on host tensors (CPU float32, ideally
    pinned): p1, p2 [n, K, 2], optional uint8 vertex counts c1, c2 [n],
    grad [n] -> (iou [n], g1, g2 [n, K, 2]) on the host.  K = 4 with every
    tensor pinned runs one kernel on the host memory in place (no workspace);
    otherwise chunked and pipelined (copies overlap the kernels).
    Asynchronous on the stream: synchronise before reading the outputs."""
    for t, name in ((p1, "p1"), (p2, "p2"), (grad, "grad")):
        if not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float32 host tensor")
    if p1.dim() != 3 or p1.shape[2] != 2 or p1.shape[1] not in (4, 8) or p2.shape != p1.shape:
        raise ValueError("p1 and p2 must be [n, K, 2] with K in (4, 8)")
    n, K = p1.shape[0], p1.shape[1]
    if grad.shape != (n,):
        raise ValueError("grad must be [n]")
    for t, name in ((c1, "c1"), (c2, "c2")):
        if t is not None and (not isinstance(t, torch.Tensor) or t.is_cuda or t.dtype != torch.uint8
                              or t.shape != (n,) or not t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous uint8 host tensor of shape [n]")
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    if out is None:
        pin = p1.is_pinned()
        out = (torch.empty(n, pin_memory=pin), torch.empty((n, K, 2), pin_memory=pin),
               torch.empty((n, K, 2), pin_memory=pin))
    iou, g1, g2 = out
    direct = (K == 4 and all(t.is_pinned() for t in (p1, p2, grad, iou, g1, g2, c1, c2) if t is not None)
              and all(t.data_ptr() % 16 == 0 for t in (p1, p2, g1, g2)))
    if workspace is None and not direct:
        workspace = torch.empty(dgal_iou_host_workspace_bytes(chunk, K) + 256, device=dev, dtype=torch.uint8)
        off = (-workspace.data_ptr()) % 256
        workspace = workspace[off:]
    ws_ptr, ws_bytes = (_lib.ptr(workspace), workspace.numel()) if workspace is not None else (None, 0)
    _lib.call("dgal_iou_fwd_bwd_host", _lib.ptr(p1), _lib.ptr(c1), _lib.ptr(p2), _lib.ptr(c2), _lib.ptr(grad), n, K,
              _lib.ptr(iou), _lib.ptr(g1), _lib.ptr(g2), ws_ptr, ws_bytes, chunk, flags, _lib.stream_ptr(stream))
    return iou, g1, g2


def dgal_nms_workspace_bytes(N, K=4):
    return int(_lib.lib().dgal_nms_workspace_bytes(N, K))


def dgal_nms_rotated(boxes, scores, threshold, counts=None, flags=DGAL_FP64_REFINE, stream=None, workspace=None,
                     sync=True):
    """Greedy rotated NMS: boxes visited by descending score (ties: lower
    index first), a box kept unless a kept box has IoU > threshold with it.
    sync=True returns the kept indices (int64 [num_keep], visiting order),
    reading the count back; sync=False returns (keep [N], num_keep [1]) on the
    device without synchronising."""
    _poly(boxes, "boxes")
    N, K = boxes.shape[0], boxes.shape[1]
    if not isinstance(scores, torch.Tensor) or scores.dtype != torch.float32 or scores.shape != (N,) \
            or scores.device != boxes.device or not scores.is_contiguous():
        raise ValueError(f"scores must be a contiguous float32 tensor of shape ({N},) on {boxes.device}")
    counts = _counts(counts, N, "counts", boxes.device)
    need = dgal_nms_workspace_bytes(N, K)
    if need == 0 and N > 0:
        raise ValueError(f"N = {N} boxes is beyond the NMS limit")
    if workspace is None:
        workspace = torch.empty(max(need, 16), device=boxes.device, dtype=torch.uint8)
    keep = torch.empty(N, device=boxes.device, dtype=torch.int64)
    num_keep = torch.empty(1, device=boxes.device, dtype=torch.int64)
    _lib.call("dgal_nms_rotated", _lib.ptr(boxes), _lib.ptr(counts), _lib.ptr(scores), N, K, float(threshold),
              _lib.ptr(keep), _lib.ptr(num_keep), _lib.ptr(workspace), workspace.numel(), flags,
              _lib.stream_ptr(stream))
    if not sync:
        return keep, num_keep
    return keep[: int(num_keep.item())]


def dgal_batched_workspace_bytes(S, K=4):
    return int(_lib.lib().dgal_batched_workspace_bytes(S, K))


def _offsets(t, S, name):
    if t.dtype != torch.int64 or t.shape != (S + 1,) or not t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name} must be a contiguous CUDA int64 tensor of shape ({S + 1},)")
    return t


def dgal_iou_pairwise_batched(a, b, a_off, b_off, out_off, total=None, ca=None, cb=None, workspace=None,
                              with_nx=True, flags=DGAL_FP64_REFINE, stream=None, out=None):
    """Ragged batch (device offsets); returns (iou packed [total], nx packed | None).

    ``total`` = out_off[S] (pass it to avoid a device->host read)."""
    _poly(a, "a")
    _poly(b, "b")
    S = a_off.shape[0] - 1
    K = a.shape[1]
    for t, nm in ((a_off, "a_off"), (b_off, "b_off"), (out_off, "out_off")):
        _offsets(t, S, nm)
    if workspace is None:
        workspace = torch.empty(dgal_batched_workspace_bytes(S, K), device=a.device, dtype=torch.uint8)
    if out is None:
        if total is None:
            total = int(out_off[-1].item())
        iou = torch.empty(total, device=a.device, dtype=torch.float32)
        nx = torch.empty(total, device=a.device, dtype=torch.uint8) if with_nx else None
    else:
        iou, nx = out
    _lib.call("dgal_iou_pairwise_batched", S, _lib.ptr(a_off), _lib.ptr(b_off), _lib.ptr(out_off), _lib.ptr(a),
              _lib.ptr(ca), _lib.ptr(b), _lib.ptr(cb), K, _lib.ptr(iou), _lib.ptr(nx), _lib.ptr(workspace),
              workspace.numel(), flags, _lib.stream_ptr(stream))
    return iou, nx


def dgal_iou_pairwise_per_scene(a, b, a_off_h, b_off_h, out_off_h, ca=None, cb=None, with_nx=True,
                                flags=DGAL_FP64_REFINE | DGAL_PLAIN, stream=None, out=None):
    """The plain form: one pairwise launch per scene (host int64 offsets, numpy or CPU tensor)."""
    import numpy as np

    _poly(a, "a")
    _poly(b, "b")
    ao = np.ascontiguousarray(a_off_h, dtype=np.int64)
    bo = np.ascontiguousarray(b_off_h, dtype=np.int64)
    oo = np.ascontiguousarray(out_off_h, dtype=np.int64)
    S = ao.shape[0] - 1
    K = a.shape[1]
    if out is None:
        iou = torch.empty(int(oo[-1]), device=a.device, dtype=torch.float32)
        nx = torch.empty(int(oo[-1]), device=a.device, dtype=torch.uint8) if with_nx else None
    else:
        iou, nx = out
    _lib.call("dgal_iou_pairwise_per_scene", S, ao.ctypes.data_as(ctypes.c_void_p),
              bo.ctypes.data_as(ctypes.c_void_p), oo.ctypes.data_as(ctypes.c_void_p), _lib.ptr(a), _lib.ptr(ca),
              _lib.ptr(b), _lib.ptr(cb), K, _lib.ptr(iou), _lib.ptr(nx), flags, _lib.stream_ptr(stream))
    return iou, nx


class BatchedGraph:
    """The ragged batch captured once into a CUDA graph; ``launch()`` replays it.

    The graph keeps the pointers of the tensors given here: rewrite them in
    place between replays, keep them alive while the graph exists."""

    def __init__(self, a, b, a_off, b_off, out_off, total, ca=None, cb=None, with_nx=True,
                 flags=DGAL_FP64_REFINE):
        _poly(a, "a")
        _poly(b, "b")
        S = a_off.shape[0] - 1
        K = a.shape[1]
        for t, nm in ((a_off, "a_off"), (b_off, "b_off"), (out_off, "out_off")):
            _offsets(t, S, nm)
        self.workspace = torch.empty(dgal_batched_workspace_bytes(S, K), device=a.device, dtype=torch.uint8)
        self.iou = torch.empty(total, device=a.device, dtype=torch.float32)
        self.nx = torch.empty(total, device=a.device, dtype=torch.uint8) if with_nx else None
        self._keep = (a, b, a_off, b_off, out_off, ca, cb)
        h = ctypes.c_void_p()
        _lib.call("dgal_batched_graph_create", ctypes.byref(h), S, _lib.ptr(a_off), _lib.ptr(b_off),
                  _lib.ptr(out_off), _lib.ptr(a), _lib.ptr(ca), _lib.ptr(b), _lib.ptr(cb), K, _lib.ptr(self.iou),
                  _lib.ptr(self.nx), _lib.ptr(self.workspace), self.workspace.numel(), flags)
        self._h = h

    def launch(self, stream=None):
        _lib.call("dgal_graph_launch", self._h, _lib.stream_ptr(stream))
        return self.iou, self.nx

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().dgal_graph_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dgal_autotune(K=4, cache_path=None, config_class=0):
    """Tune a launch shape (0: the ragged batch, 1: the paired calls); returns
    the shape now in use (dgal_get_batched_config / dgal_get_paired_config)."""
    _lib.call("dgal_autotune", K, config_class, None if cache_path is None else str(cache_path).encode())
    return dgal_get_batched_config(K) if config_class == 0 else dgal_get_paired_config(K)


def dgal_get_paired_config(K=4):
    out = ctypes.c_int64(0)
    _lib.call("dgal_get_paired_config", K, ctypes.byref(out))
    return dict(group_below=out.value)


def dgal_get_batched_config(K=4):
    out = (ctypes.c_int32 * 3)()
    _lib.call("dgal_get_batched_config", K, out)
    return dict(tile=out[0], threads=out[1], blocks_per_sm=out[2])


def dgal_get_device_status(clear=False):
    v = ctypes.c_uint32(0)
    _lib.call("dgal_get_device_status", ctypes.byref(v), 1 if clear else 0)
    return v.value


def dgal_last_error():
    return _lib.lib().dgal_last_error().decode(errors="replace")


def dgal_version():
    return int(_lib.lib().dgal_version())


# Memory budget of the saved flags of ``IoU`` (bytes): above it the forward
# keeps no flags and the backward re-runs the clip.  The flags take 1 + 2K
# bytes per pair (9 for quadrilaterals: 90 MB for 10^7 pairs, 170 MB for
# K = 8).  Overridden by the environment variable DGAL_FLAG_BUDGET_BYTES or
# by IoU's ``flag_budget`` argument.
DEFAULT_FLAG_BUDGET_BYTES = 64 << 20


def flag_budget_bytes(budget=None):
    """The flag budget in bytes: ``budget`` if given, else
    DGAL_FLAG_BUDGET_BYTES from the environment, else the default (64 MiB)."""
    if budget is not None:
        return int(budget)
    env = os.environ.get("DGAL_FLAG_BUDGET_BYTES")
    return int(env) if env else DEFAULT_FLAG_BUDGET_BYTES


def choose_recompute(n, K, recompute=None, budget=None):
    """Recompute mode for n pairs of capacity K: ``recompute`` when given,
    else True exactly when the saved flags (n (1 + 2K) bytes) would exceed the
    flag budget."""
    if recompute is not None:
        return bool(recompute)
    return n * (1 + 2 * K) > flag_budget_bytes(budget)


class IoU(torch.autograd.Function):
    """IoU of paired convex polygons with the library's hand-written backward.

    Saved-flag mode records (nx, xflags) in the forward (1 + 2K bytes per
    pair) and the backward reads them; recompute mode stores nothing and the
    backward re-runs the clip.  ``recompute=None`` picks recompute mode when
    the flags would exceed the flag budget (``choose_recompute``)."""

    @staticmethod
    def forward(ctx, p1, p2, c1=None, c2=None, recompute=None, flags=DGAL_FP64_REFINE, flag_budget=None):
        p1c, p2c = p1.contiguous(), p2.contiguous()
        recompute = choose_recompute(p1c.shape[0], p1c.shape[1], recompute, flag_budget)
        ctx.recompute = recompute
        iou_v, nx, xflags, _ = dgal_iou_paired(p1c, p2c, c1, c2, save_flags=not recompute, flags=flags)
        ctx.save_for_backward(p1c, p2c, nx, xflags, c1, c2)
        ctx.flags = flags
        return iou_v

    @staticmethod
    def backward(ctx, grad):
        p1, p2, nx, xflags, c1, c2 = ctx.saved_tensors
        g1, g2 = dgal_iou_backward(p1, p2, grad.contiguous().float(), nx, xflags, c1, c2, flags=ctx.flags)
        return g1, g2, None, None, None, None, None


def iou(p1, p2, c1=None, c2=None, recompute=None, flags=DGAL_FP64_REFINE, flag_budget=None):
    """Differentiable paired IoU (see ``IoU``)."""
    return IoU.apply(p1, p2, c1, c2, recompute, flags, flag_budget)


class IoULoss(torch.autograd.Function):
    """loss = scale * sum w (1 - IoU) (or GIoU / DIoU) through dgal_iou_loss:
    the forward computes the loss and keeps the clip state in a workspace; the
    backward runs dgal_iou_loss_backward on it with the incoming gradient
    read on the device (no arithmetic outside the library)."""

    @staticmethod
    def forward(ctx, p1, p2, weight=None, scale=1.0, c1=None, c2=None, flags=DGAL_FP64_REFINE, variant="iou"):
        p1c, p2c = p1.contiguous(), p2.contiguous()
        n, K = p1c.shape[0], p1c.shape[1]
        ws = torch.empty(max(dgal_iou_loss_workspace_bytes(n, K), 16), device=p1c.device, dtype=torch.uint8)
        loss, _, _, _ = dgal_iou_loss(p1c, p2c, weight, scale, c1, c2, grads=False, flags=flags, workspace=ws,
                                      variant=variant)
        ctx.save_for_backward(p1c, p2c, weight, c1, c2, ws)
        ctx.scale, ctx.flags, ctx.variant = scale, flags, variant
        return loss[0]

    @staticmethod
    def backward(ctx, grad):
        p1, p2, weight, c1, c2, ws = ctx.saved_tensors
        g1, g2 = dgal_iou_loss_backward(p1, p2, ws, grad.reshape(1).float(), weight, ctx.scale, c1, c2,
                                        flags=ctx.flags, variant=ctx.variant)
        return g1, g2, None, None, None, None, None, None


def iou_loss(p1, p2, weight=None, reduction="sum", c1=None, c2=None, flags=DGAL_FP64_REFINE, variant="iou"):
    """Differentiable IoU loss sum_k w_k (1 - IoU_k) (or its mean over pairs);
    variant "giou" / "diou" for the generalized / distance IoU loss."""
    if reduction not in ("sum", "mean"):
        raise ValueError("reduction must be 'sum' or 'mean'")
    scale = 1.0 / max(p1.shape[0], 1) if reduction == "mean" else 1.0
    return IoULoss.apply(p1, p2, weight, scale, c1, c2, flags, variant)


class IoU3D(torch.autograd.Function):
    """3D IoU of paired boxes (bird's-eye-view polygon + (z_center, height))
    with the hand-written backward; the flags of the forward are saved."""

    @staticmethod
    def forward(ctx, p1, z1, p2, z2, c1=None, c2=None, flags=DGAL_FP64_REFINE):
        p1c, p2c, z1c, z2c = p1.contiguous(), p2.contiguous(), z1.contiguous(), z2.contiguous()
        iou_v, nx, xflags, _ = dgal_iou3d_paired(p1c, z1c, p2c, z2c, c1, c2, flags=flags)
        ctx.save_for_backward(p1c, z1c, p2c, z2c, nx, xflags, c1, c2)
        ctx.flags = flags
        return iou_v

    @staticmethod
    def backward(ctx, grad):
        p1, z1, p2, z2, nx, xflags, c1, c2 = ctx.saved_tensors
        g1, gz1, g2, gz2 = dgal_iou3d_backward(p1, z1, p2, z2, grad.contiguous().float(), nx, xflags, c1, c2,
                                               flags=ctx.flags)
        return g1, gz1, g2, gz2, None, None, None


def iou3d(p1, z1, p2, z2, c1=None, c2=None, flags=DGAL_FP64_REFINE):
    """Differentiable paired 3D IoU (see ``IoU3D``)."""
    return IoU3D.apply(p1, z1, p2, z2, c1, c2, flags)


class IoU3DLoss(torch.autograd.Function):
    """loss = scale * sum w (1 - IoU3) through dgal_iou3d_loss; the backward
    runs dgal_iou3d_loss_backward with the incoming gradient read on the
    device."""

    @staticmethod
    def forward(ctx, p1, z1, p2, z2, weight=None, scale=1.0, c1=None, c2=None, flags=DGAL_FP64_REFINE):
        ts = [t.contiguous() for t in (p1, z1, p2, z2)]
        n, K = ts[0].shape[0], ts[0].shape[1]
        ws = torch.empty(max(dgal_iou_loss_workspace_bytes(n, K), 16), device=ts[0].device, dtype=torch.uint8)
        loss, *_ = dgal_iou3d_loss(*ts, weight, scale, c1, c2, grads=False, flags=flags, workspace=ws)
        ctx.save_for_backward(*ts, weight, c1, c2, ws)
        ctx.scale, ctx.flags = scale, flags
        return loss[0]

    @staticmethod
    def backward(ctx, grad):
        p1, z1, p2, z2, weight, c1, c2, ws = ctx.saved_tensors
        g1, gz1, g2, gz2 = dgal_iou3d_loss_backward(p1, z1, p2, z2, ws, grad.reshape(1).float(), weight, ctx.scale,
                                                    c1, c2, flags=ctx.flags)
        return (g1, gz1, g2, gz2) + (None,) * 5


def iou3d_loss(p1, z1, p2, z2, weight=None, reduction="sum", c1=None, c2=None, flags=DGAL_FP64_REFINE):
    """Differentiable 3D IoU loss sum_k w_k (1 - IoU3_k) (or its mean over pairs)."""
    if reduction not in ("sum", "mean"):
        raise ValueError("reduction must be 'sum' or 'mean'")
    scale = 1.0 / max(p1.shape[0], 1) if reduction == "mean" else 1.0
    return IoU3DLoss.apply(p1, z1, p2, z2, weight, scale, c1, c2, flags)
