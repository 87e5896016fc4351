"""The GPU forward's rule for exactly zero orientations, modelled on the host
in exact rational arithmetic.

With refinement, an orientation that is exactly zero (a vertex on the line of
an edge: shared edges, touching vertices) takes the sign it has when P2 is
translated by an infinitesimal (eps, eps^2): a zero S(i,j) = orient(b_j,
b_j+1, a_i) takes the sign of eby_j (of -ebx_j when eby_j = 0), a zero T(i,j)
= orient(a_i, a_i+1, b_j) the sign of -eay_i (of eax_i when eay_i = 0).  The
pins here:
  * the rule equals the signs of an actual translation by (eps, eps^2) with a
    tiny rational eps, on every orientation of constructed shared-edge and
    touching-vertex pairs (and a wrong rule does not);
  * with those signs every pair is in general position: the inside tests and
    proper crossings give a valid boundary walk (the same walk as the
    kernel's), and
  * the kernel's area formula over that walk's terms, evaluated at eps = 0,
    equals the exact area of the clip (Sutherland-Hodgman in fractions) of
    the untranslated pair;
  * the group forward's second pass (every zero's sign flipped) is the
    opposite translation, and one of the two leaves every shared-edge and
    touching-vertex pair with an empty clip.
"""
from fractions import Fraction as F

import numpy as np
import pytest

from paper_2011_11134_gb300 import workloads as W

from .exact_clip import area as exact_area, clip as exact_clip


def _cross(ux, uy, vx, vy):
    return ux * vy - uy * vx


def tie_neg(ex, ey, p1edge):
    """The kernel's rule: negative sign of a zero orientation, from the edge
    vector (ex, ey) of the edge's polygon (P1 for a T orientation)."""
    if ey != 0:
        return (ey > 0) == p1edge
    if ex != 0:
        return (ex < 0) == p1edge
    return None


def signs(p, q, n1, n2, rule=tie_neg):
    """Exact S, T and the negative-sign matrices after the tie rule."""
    A = [(F(float(x)), F(float(y))) for x, y in p[:n1]]
    B = [(F(float(x)), F(float(y))) for x, y in q[:n2]]
    ea = [(A[(i + 1) % n1][0] - A[i][0], A[(i + 1) % n1][1] - A[i][1]) for i in range(n1)]
    eb = [(B[(j + 1) % n2][0] - B[j][0], B[(j + 1) % n2][1] - B[j][1]) for j in range(n2)]
    S = [[_cross(*eb[j], A[i][0] - B[j][0], A[i][1] - B[j][1]) for j in range(n2)] for i in range(n1)]
    T = [[_cross(*ea[i], B[j][0] - A[i][0], B[j][1] - A[i][1]) for j in range(n2)] for i in range(n1)]
    nS = [[(S[i][j] < 0) if S[i][j] != 0 else rule(*eb[j], False) for j in range(n2)] for i in range(n1)]
    nT = [[(T[i][j] < 0) if T[i][j] != 0 else rule(*ea[i], True) for j in range(n2)] for i in range(n1)]
    return A, B, ea, eb, S, T, nS, nT


def translated_neg(A, B, n1, n2, eps, sign=1):
    """Negative-sign matrices of the pair with P2 translated by sign (eps, eps^2)."""
    Bt = [(x + sign * eps, y + sign * eps * eps) for x, y in B]
    ea = [(A[(i + 1) % n1][0] - A[i][0], A[(i + 1) % n1][1] - A[i][1]) for i in range(n1)]
    eb = [(Bt[(j + 1) % n2][0] - Bt[j][0], Bt[(j + 1) % n2][1] - Bt[j][1]) for j in range(n2)]
    S = [[_cross(*eb[j], A[i][0] - Bt[j][0], A[i][1] - Bt[j][1]) for j in range(n2)] for i in range(n1)]
    T = [[_cross(*ea[i], Bt[j][0] - A[i][0], Bt[j][1] - A[i][1]) for j in range(n2)] for i in range(n1)]
    assert all(v != 0 for row in S + T for v in row), "the translated pair is in general position"
    return [[v < 0 for v in row] for row in S], [[v < 0 for v in row] for row in T]


def walk_and_area(A, B, ea, eb, S, T, nS, nT, n1, n2):
    """The kernel's boundary walk and select-free area from the sign matrices
    (no value is compared with zero here), in P1's local frame."""
    o = A[0]
    a = [(x - o[0], y - o[1]) for x, y in A]
    b = [(x - o[0], y - o[1]) for x, y in B]
    sp = [[not nS[i][j] for j in range(n2)] for i in range(n1)]
    tp = [[not nT[i][j] for j in range(n2)] for i in range(n1)]
    in1 = [all(sp[i]) for i in range(n1)]
    in2 = [all(tp[i][j] for i in range(n1)) for j in range(n2)]
    X = [[sp[i][j] != sp[(i + 1) % n1][j] and tp[i][j] != tp[i][(j + 1) % n2] for j in range(n2)]
         for i in range(n1)]
    # P2 leaves P1 exactly where P1 enters P2 (the kernel's consistency check)
    for i in range(n1):
        for j in range(n2):
            if X[i][j]:
                assert tp[i][j] == (not sp[i][j])
    seq = []
    for i in range(n1):
        if in1[i]:
            seq.append(i)
        ent = [j for j in range(n2) if X[i][j] and not sp[i][j]]
        ext = [j for j in range(n2) if X[i][j] and sp[i][j]]
        assert len(ent) <= 1 and len(ext) <= 1
        if ent:
            seq.append(0x80 | (i << 3) | ent[0])
        if ext:
            seq.append(0x80 | (i << 3) | ext[0])
            j = (ext[0] + 1) % n2
            while in2[j]:
                seq.append(0x40 | j)
                j = (j + 1) % n2
    nX = sum(map(sum, X))
    if nX == 0 and not any(in1):
        seq = [0x40 | j for j in range(n2)] if all(in2) else []
    assert len(seq) == len(set(seq)), "no code twice"
    assert len(seq) == sum(in1) + sum(in2) + nX or (not seq and nX == 0)
    two_a = F(0)
    if seq:
        for v in range(n1):
            if in1[(v + 1) % n1]:
                two_a += _cross(*a[v], *ea[v])
        for v in range(n2):
            if in2[(v + 1) % n2]:
                two_a += _cross(*b[v], *eb[v])
        for i in range(n1):
            for j in range(n2):
                if X[i][j]:
                    D = _cross(*ea[i], *eb[j])
                    assert D != 0, "no crossing of parallel edges"
                    two_a += (_cross(*a[i], *b[j]) * D + S[i][j] * T[i][j]) / abs(D)
    return seq, two_a / 2


def _pairs(n=400, seed=31):
    d = W.convex_pairs_4m(seed=seed, n=n, degenerate_frac=1.0)
    keep = (d["kind"] == 2) | (d["kind"] == 3)
    return [(d["p1"][k], d["p2"][k], int(d["c1"][k]), int(d["c2"][k]), int(d["kind"][k]))
            for k in np.nonzero(keep)[0]]


def test_rule_is_a_translation():
    eps = F(1, 10 ** 40)
    zeros = 0
    for p, q, n1, n2, kind in _pairs():
        A, B, ea, eb, S, T, nS, nT = signs(p, q, n1, n2)
        zeros += sum(v == 0 for row in S + T for v in row)
        tS, tT = translated_neg(A, B, n1, n2, eps)
        assert nS == tS and nT == tT, (kind, n1, n2)
    assert zeros > 300, "the constructed pairs have exact zeros"


def test_wrong_rule_is_not_a_translation():
    """A rule with the S and T cases swapped disagrees with the translation."""
    def swapped(ex, ey, p1edge):
        return tie_neg(ex, ey, not p1edge)
    eps = F(1, 10 ** 40)
    differ = 0
    for p, q, n1, n2, kind in _pairs(n=120):
        A, B, ea, eb, S, T, nS, nT = signs(p, q, n1, n2, rule=swapped)
        tS, tT = translated_neg(A, B, n1, n2, eps)
        differ += (nS != tS) or (nT != tT)
    assert differ > 10


@pytest.mark.parametrize("seed", [31, 32])
def test_walk_area_equals_exact_clip(seed):
    checked = empty = 0
    for p, q, n1, n2, kind in _pairs(n=300, seed=seed):
        A, B, ea, eb, S, T, nS, nT = signs(p, q, n1, n2)
        seq, a = walk_and_area(A, B, ea, eb, S, T, nS, nT, n1, n2)
        inter = exact_clip(p[:n1].tolist(), q[:n2].tolist())
        ref = exact_area(inter) if len(inter) >= 3 else F(0)
        assert a == ref, (kind, float(a), float(ref))
        checked += 1
        empty += not seq
    # shared edges and touching vertices have no area; the walk finds either an
    # empty intersection or a sliver of zero area, depending on the side the
    # translation moves P2 to
    assert checked > 100 and 0 < empty < checked


def test_opposite_translation_empties_touching_pairs():
    eps = F(1, 10 ** 40)
    second = 0
    for p, q, n1, n2, kind in _pairs(n=300, seed=33):
        A, B, ea, eb, S, T, nS, nT = signs(p, q, n1, n2)
        seq, a = walk_and_area(A, B, ea, eb, S, T, nS, nT, n1, n2)
        if not seq:
            continue
        # the second pass: every zero orientation's sign flipped
        fS = [[(not nS[i][j]) if S[i][j] == 0 else nS[i][j] for j in range(n2)] for i in range(n1)]
        fT = [[(not nT[i][j]) if T[i][j] == 0 else nT[i][j] for j in range(n2)] for i in range(n1)]
        tS, tT = translated_neg(A, B, n1, n2, eps, sign=-1)
        assert fS == tS and fT == tT, "the flipped signs are the opposite translation's"
        seq2, a2 = walk_and_area(A, B, ea, eb, S, T, fS, fT, n1, n2)
        assert seq2 == [] and a2 == 0, (kind, seq2)
        second += 1
    assert second > 30
