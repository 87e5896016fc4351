"""Shared helpers of the GPU parity tests (comparison rules, tolerances)."""
import os

import numpy as np

# Parity bar: IoU within 1e-5 absolute of the FP64 oracle on every pair;
# gradients within 1e-3 relative (per pair, max |dg| / max(max |g_ref|, 1e-6))
# on pairs neither side flags near-degenerate; nx / xflags bit-exact there.
IOU_ATOL = 1e-5
GRAD_RTOL = 1e-3

THREADS = max(1, min(16, os.cpu_count() or 1))


def dev(x, device="cuda"):
    import torch

    return torch.from_numpy(np.ascontiguousarray(x)).to(device)


def host(t):
    return t.detach().cpu().numpy()


def check_forward(iou, nx, xflags, degen, ref, label=""):
    """Returns the generic mask after asserting the parity bar."""
    iou = iou.astype(np.float64)
    err = np.abs(iou - ref["iou"])
    assert err.max() <= IOU_ATOL, f"{label}: max IoU error {err.max():.3e} at {int(err.argmax())}"
    generic = (ref["degen"] == 0)
    if degen is not None:
        generic &= (degen & 1) == 0
    if nx is not None:
        bad = np.nonzero((nx != ref["nx"]) & generic)[0]
        assert bad.size == 0, f"{label}: nx mismatch on {bad.size} generic pairs, first {bad[:5]}"
    if xflags is not None:
        bad = np.nonzero((xflags != ref["xflags"]).any(1) & generic)[0]
        assert bad.size == 0, (f"{label}: xflags mismatch on {bad.size} generic pairs, first {bad[:5]}: "
                               f"{xflags[bad[:3]]} vs {ref['xflags'][bad[:3]]}")
    return generic


def grad_rel_err(g1, g2, r1, r2, mask):
    G = np.concatenate([g1, g2], 1).astype(np.float64)[mask]
    R = np.concatenate([r1, r2], 1)[mask]
    if G.shape[0] == 0:
        return np.zeros(0)
    return np.abs(G - R).max(axis=(1, 2)) / np.maximum(np.abs(R).max(axis=(1, 2)), 1e-6)
