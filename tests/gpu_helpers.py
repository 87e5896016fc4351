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


def check_flagged_grads(g1, g2, p1, p2, c1, c2, ref, mask, grad=None, label=""):
    """Gradients of the pairs in `mask` (those the parity bar waives: near-
    degenerate on either side) are still finite and bounded by what the IoU
    allows.  dIoU = dA_i (A_1 + A_2) / U^2 - (A_i / U^2)(dA_1 + dA_2), with
    (A_1 + A_2) / U^2 <= 2 / U and A_i / U^2 <= 1 / U; a vertex moves each area
    at most by the length of its two incident edge pieces over 2, i.e. by at
    most the diameter 2 sqrt(2) L of the pair (L the largest |coordinate|
    about P1's vertex 0).  So |dIoU/dv| <= 3 * 2 sqrt(2) L / U; the check
    allows twice that."""
    idx = np.nonzero(mask)[0]
    if idx.size == 0:
        return
    G = np.concatenate([g1[idx], g2[idx]], 1).astype(np.float64)
    assert np.isfinite(G).all(), f"{label}: non-finite gradient on a flagged pair"
    P = np.concatenate([p1[idx], p2[idx]], 1).astype(np.float64)
    if c1 is not None:
        K = p1.shape[1]
        live = np.concatenate([np.arange(K)[None, :] < c1[idx, None], np.arange(K)[None, :] < c2[idx, None]], 1)
        P = np.where(live[..., None], P, P[:, :1])
    L = np.abs(P - P[:, :1]).max(axis=(1, 2))
    U = ref["areas"][idx, 1] + ref["areas"][idx, 2] - ref["areas"][idx, 0]
    up = np.ones(idx.size) if grad is None else np.abs(np.asarray(grad, np.float64)[idx])
    ok = U > 1e-12 * np.maximum(L, 1e-30) ** 2
    bound = 2.0 * 3.0 * 2.0 * np.sqrt(2.0) * L / np.where(ok, U, 1.0) * up
    gmax = np.abs(G).max(axis=(1, 2))
    bad = np.nonzero(ok & (gmax > bound))[0]
    assert bad.size == 0, f"{label}: gradient above the IoU bound on {bad.size} flagged pairs, first {idx[bad[:5]]}"
