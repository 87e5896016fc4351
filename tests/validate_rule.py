"""The input check of DGAL_VALIDATE / dgal_validate_polygons, stated on the
host in exact rational arithmetic, and the polygon families the tests feed it.

A polygon (its first m vertices) passes when every vertex lies strictly left
of every edge it is not an end of.  The CPU test pins that rule to an
independent characterisation (the polygon is its own strict convex hull, in
counter-clockwise order); the GPU test compares the kernel with it.
"""
from fractions import Fraction as F

import numpy as np


def _orient(a, b, p):
    return (b[0] - a[0]) * (p[1] - a[1]) - (b[1] - a[1]) * (p[0] - a[0])


def passes(poly, m):
    """The kernel's rule on the float32 vertices, exactly."""
    v = [(F(float(x)), F(float(y))) for x, y in poly[:m]]
    for i in range(m):
        a, b = v[i], v[(i + 1) % m]
        for k in range(m):
            if k in (i, (i + 1) % m):
                continue
            if _orient(a, b, v[k]) <= 0:
                return False
    return True


def strict_hull_ccw(pts):
    """Andrew's monotone chain on exact points, collinear points dropped:
    the strict convex hull, counter-clockwise from the lowest-leftmost point."""
    P = sorted(set(pts))
    if len(P) < 3:
        return P
    lower, upper = [], []
    for p in P:
        while len(lower) >= 2 and _orient(lower[-2], lower[-1], p) <= 0:
            lower.pop()
        lower.append(p)
    for p in reversed(P):
        while len(upper) >= 2 and _orient(upper[-2], upper[-1], p) <= 0:
            upper.pop()
        upper.append(p)
    return lower[:-1] + upper[:-1]


def is_own_strict_hull(poly, m):
    """Independent form: the m vertices are distinct, all on the strict hull,
    and in the hull's counter-clockwise cyclic order."""
    v = [(F(float(x)), F(float(y))) for x, y in poly[:m]]
    if len(set(v)) != m:
        return False
    h = strict_hull_ccw(v)
    if len(h) != m:
        return False
    s = h.index(v[0])
    return h[s:] + h[:s] == v


def families(seed=5, n=300):
    """float32 [N, 8, 2] polygons with counts, and the family name of each:
    valid hulls and quads, and broken copies (clockwise, two vertices swapped,
    a vertex moved inward, exact collinear and repeated vertices, vertices
    nudged just outside or inside the line of their neighbours)."""
    from paper_2011_11134_gb300 import workloads as W

    r = np.random.Generator(np.random.PCG64(seed))
    d = W.convex_pairs_4m(seed=seed, n=n, degenerate_frac=0.0)
    hulls, cnt = d["p1"].astype(np.float32), d["c1"].astype(np.int64)
    quads = W.loss_pairs_1m(seed=seed, n=n)["p1"].astype(np.float32)
    out, counts, names = [], [], []

    def add(p, m, name):
        q = np.zeros((8, 2), np.float32)
        q[:m] = p[:m]
        q[m:] = p[0]
        out.append(q)
        counts.append(m)
        names.append(name)

    for k in range(n):
        m = int(cnt[k])
        h = hulls[k]
        add(h, m, "hull")
        add(quads[k], 4, "quad")
        add(h[:m][::-1], m, "clockwise")
        q = quads[k].copy()
        q[[1, 2]] = q[[2, 1]]
        add(q, 4, "bowtie")
        if m >= 4:
            # v1 moved across the chord v0 v2, to its left (the polygon's side):
            # the turn at v1 is then a right turn
            g = h[:m].astype(np.float64)
            e = g[2] - g[0]
            g[1] = 0.5 * (g[0] + g[2]) + 0.1 * np.array([-e[1], e[0]])
            add(g.astype(np.float32), m, "reflex")
        g = h[:m].copy()
        g[1] = g[0]
        add(g, m, "repeated")
        # v1 just off the line v0 v2, by a few ulps of the coordinates, either side
        g = h[:m].astype(np.float64)
        e = g[2] - g[0]
        nrm = np.array([e[1], -e[0]]) / np.linalg.norm(e)  # outward for a CCW polygon
        side = r.choice([-1.0, 1.0])
        g[1] = 0.5 * (g[0] + g[2]) + side * r.uniform(1e-7, 1e-5) * np.abs(g).max() * nrm
        add(g.astype(np.float32), m, "nudged")
    # exactly collinear vertices on an axis-aligned outline
    for s in (1.0, 0.25, 1024.0):
        add(np.array([[0, 0], [1, 0], [2, 0], [2, 2], [0, 2]], np.float32) * s, 5, "collinear")
        add(np.array([[0, 0], [2, 0], [2, 2], [0, 2]], np.float32) * s + 3, 4, "square")
    # a pentagram: every turn is a left turn, but the outline winds twice
    t = 2 * np.pi * np.arange(5) / 5
    star = np.stack([np.cos(2 * t), np.sin(2 * t)], 1).astype(np.float32)
    add(star, 5, "pentagram")
    return np.stack(out), np.array(counts, np.uint8), names
