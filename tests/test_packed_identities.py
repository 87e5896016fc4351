"""The rewritten forms the packed-pair kernels evaluate, against the plain
definitions, in FP64 on random local-frame geometry.

The packed blocks (two P2 edges per f32x2 instruction) form, with the
differences mx = bx_j - ax_i and dy = ay_i - by_j,
    S  = ebx_j dy + eby_j mx          = orient(b_j, b_j+1, a_i),
    nT = eax_i dy + eay_i mx          = -orient(a_i, a_i+1, b_j),
    D  = eax_i eby_j - eay_i ebx_j    = cross(ea_i, eb_j),
    nc = ay_i bx_j - ax_i by_j        = -cross(a_i, b_j),
and the forward's crossing term of the area as (nc D + S nT) / (-|D|), which
must equal (cross(a_i, b_j) D + S T) / |D|.  The signs of T come from nT
inverted.  A slip in any of these conventions fails here.
"""
import numpy as np


def _cross(ux, uy, vx, vy):
    return ux * vy - uy * vx


def _orient(ax, ay, bx, by, px, py):
    return _cross(bx - ax, by - ay, px - ax, py - ay)


def test_packed_block_forms_equal_definitions():
    r = np.random.Generator(np.random.PCG64(3))
    n = 20000
    a, a1, b, b1 = (r.uniform(-5, 5, size=(n, 2)) for _ in range(4))
    ax, ay = a.T
    bx, by = b.T
    eax, eay = (a1 - a).T
    ebx, eby = (b1 - b).T
    mx, dy = bx - ax, ay - by
    S = ebx * dy + eby * mx
    nT = eax * dy + eay * mx
    D = eax * eby - eay * ebx
    nc = ay * bx - ax * by
    S_def = _orient(bx, by, b1[:, 0], b1[:, 1], ax, ay)
    T_def = _orient(ax, ay, a1[:, 0], a1[:, 1], bx, by)
    D_def = _cross(eax, eay, ebx, eby)
    c_def = _cross(ax, ay, bx, by)
    scale = 1e-12 * 100.0
    assert np.abs(S - S_def).max() <= scale
    assert np.abs(nT + T_def).max() <= scale
    assert np.abs(D - D_def).max() <= scale
    assert np.abs(nc + c_def).max() <= scale
    term = (nc * D + S * nT) / (-np.abs(D))
    term_def = (c_def * D_def + S_def * T_def) / np.abs(D_def)
    assert np.allclose(term, term_def, rtol=1e-9, atol=1e-9)
    # the sign bits of -T, inverted, are those of T wherever T is not zero
    assert ((nT < 0) == (T_def > 0)).all()


def test_backward_crossing_parameters():
    """The backward's t = S / D and u = (-T) / D are the crossing parameters:
    a_i + t ea_i = b_j + u eb_j (the crossing point of the two lines)."""
    r = np.random.Generator(np.random.PCG64(4))
    n = 20000
    a, a1, b, b1 = (r.uniform(-5, 5, size=(n, 2)) for _ in range(4))
    ea, eb = a1 - a, b1 - b
    mx, dy = b[:, 0] - a[:, 0], a[:, 1] - b[:, 1]
    S = eb[:, 0] * dy + eb[:, 1] * mx
    nT = ea[:, 0] * dy + ea[:, 1] * mx
    D = ea[:, 0] * eb[:, 1] - ea[:, 1] * eb[:, 0]
    keep = np.abs(D) > 1e-3
    t, u = S[keep] / D[keep], nT[keep] / D[keep]
    pa = a[keep] + t[:, None] * ea[keep]
    pb = b[keep] + u[:, None] * eb[keep]
    assert np.abs(pa - pb).max() <= 1e-7
