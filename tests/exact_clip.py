"""Exact rational polygon clipping, used only to pin the oracle.

Sutherland-Hodgman clipping of P1 by each half-plane of P2 in
``fractions.Fraction`` arithmetic over the exact values of the float inputs.
This is a different algorithm from the oracle's (candidate gathering plus an
angular sort in double), and it has no rounding at all, so its area is the
exact area of P1 ∩ P2 for the given inputs.

Provenance codes are recovered geometrically from the exact vertices, with
the same precedence the method states for coincident points (P1 vertex, then
P2 vertex, then edge crossing), so the canonical flag sequence can be checked
without trusting any floating-point decision.
"""
from __future__ import annotations

from fractions import Fraction as F


def _fr(poly):
    return [(F(float(x)), F(float(y))) for x, y in poly]


def _orient(a, b, p):
    return (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0])


def clip(p1, p2):
    """Exact intersection polygon of convex CCW p1, p2 (lists of (x, y))."""
    P = _fr(p1)
    Q = _fr(p2)
    out = P
    for j in range(len(Q)):
        c, d = Q[j], Q[(j + 1) % len(Q)]
        inp, out = out, []
        if not inp:
            break
        for k in range(len(inp)):
            s, e = inp[k], inp[(k + 1) % len(inp)]
            fs, fe = _orient(c, d, s), _orient(c, d, e)
            if fs >= 0:
                out.append(s)
            if (fs > 0 and fe < 0) or (fs < 0 and fe > 0):
                t = fs / (fs - fe)
                out.append((s[0] + t * (e[0] - s[0]), s[1] + t * (e[1] - s[1])))
    # drop consecutive duplicates
    res = []
    for v in out:
        if not res or res[-1] != v:
            res.append(v)
    while len(res) > 1 and res[0] == res[-1]:
        res.pop()
    return res


def area(poly):
    poly = [(p[0] if isinstance(p[0], F) else F(float(p[0])), p[1] if isinstance(p[1], F) else F(float(p[1])))
            for p in poly]
    s = F(0)
    n = len(poly)
    for k in range(n):
        s += poly[k][0] * poly[(k + 1) % n][1] - poly[k][1] * poly[(k + 1) % n][0]
    return s / 2


def _on_segment(a, b, p):
    if _orient(a, b, p) != 0:
        return False
    return min(a[0], b[0]) <= p[0] <= max(a[0], b[0]) and min(a[1], b[1]) <= p[1] <= max(a[1], b[1])


def codes(p1, p2, inter):
    """Canonical code sequence of an exact intersection polygon, or None if a
    vertex cannot be attributed (degenerate input)."""
    P, Q = _fr(p1), _fr(p2)
    seq = []
    for v in inter:
        code = None
        for i, p in enumerate(P):
            if p == v:
                code = i
                break
        if code is None:
            for j, q in enumerate(Q):
                if q == v:
                    code = 0x40 | j
                    break
        if code is None:
            hits = [(i, j) for i in range(len(P)) for j in range(len(Q))
                    if _on_segment(P[i], P[(i + 1) % len(P)], v) and _on_segment(Q[j], Q[(j + 1) % len(Q)], v)]
            if len(hits) != 1:
                return None
            i, j = hits[0]
            code = 0x80 | (i << 3) | j
        seq.append(code)
    if len(seq) < 3:
        return []
    s0 = seq.index(min(seq))
    return seq[s0:] + seq[:s0]
