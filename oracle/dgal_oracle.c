/*
 * FP64 CPU oracle for convex-polygon intersection-over-union and its gradient
 * (DGAL, "Differentiable Computational Geometry for 2D and 3D machine
 * learning", arXiv:2011.11134).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline / reference arm may load this library.  The
 * product path (the CUDA library and its Python binding) never calls it and
 * shares no code with it.
 *
 * What it computes (paper Sec. II-B listing, `iou` and `iou_backward`):
 *   IoU(P1, P2) = A_i / (A_1 + A_2 - A_i), where A_i is the area of the
 *   intersection polygon P1 ∩ P2 (`intersect`, `area`), A_1, A_2 the areas of
 *   the inputs; `nx` is the vertex count of the intersection polygon and
 *   `xflags` records where each of its vertices comes from, so that the
 *   backward can map dL/dIoU onto the input vertices without re-clipping.
 * Polygons are convex, counter-clockwise, stored in a fixed-capacity point
 * array (paper Sec. II-C and Sec. III "(Convex) Polygons"); gradients have
 * the shape of the polygons (Sec. III, last paragraph).
 *
 * The paper leaves the clipping algorithm, the flag encoding, the vertex
 * order and degenerate handling open.  This file fixes them as follows
 * (plain definitions, written out without any blocking or fusion):
 *   - candidates: every P1 vertex inside-or-on P2 (orient >= 0 for all P2
 *     edges); every P2 vertex inside-or-on P1 that is not bit-identical to a
 *     P1 vertex; every proper crossing of a P1 edge with a P2 edge
 *     (D != 0, 0 < t < 1, 0 < u < 1);
 *   - the intersection polygon is these points in counter-clockwise order
 *     (sorted by atan2 about their centroid), rotated so the smallest code
 *     comes first;
 *   - codes: P1 vertex i -> i, P2 vertex j -> 0x40|j, crossing of P1 edge i
 *     with P2 edge j -> 0x80|(i<<3)|j, unused slots -> 0xFF;
 *   - fewer than three candidates -> empty intersection (nx = 0, IoU = 0).
 * The backward is the shoelace adjoint over the ordered vertices, routed by
 * code: vertex codes go straight to that vertex, crossing codes go through
 * the adjoint of P = a + t r, t = cross(c-a, s) / cross(r, s).
 *
 * All arithmetic is IEEE double with no contraction (built with
 * -ffp-contract=off so x86 and Arm give identical results).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXK 8
#define ORC_MAXC (2 * ORC_MAXK)
#define ORC_MAXCAND (ORC_MAXK + ORC_MAXK + ORC_MAXK * ORC_MAXK)

/* Relative threshold of the near-degenerate classifier. */
#define ORC_DEGEN_REL 1e-5

/* Status bits returned by the per-pair routines. */
#define ORC_ST_BAD_COUNT 1   /* vertex count outside [3, K] */
#define ORC_ST_OVERFLOW 2    /* more candidates than K1 + K2 slots */

typedef struct {
    double x, y;
} opt;

typedef struct {
    opt p;
    uint8_t code;
    double ang;
} ocand;

/* Per-pair forward result (w: the intersection polygon's vertices, in the
 * order of code). */
typedef struct {
    double iou, ai, a1, a2;
    int nx;
    uint8_t code[ORC_MAXC];
    opt w[ORC_MAXC];
    int degen;
    int status;
} ofwd;

static double cross2(opt a, opt b) { return a.x * b.y - a.y * b.x; }
static opt sub2(opt a, opt b) { opt r = {a.x - b.x, a.y - b.y}; return r; }

/* orient(a, b, p) > 0 when p is left of the directed line a -> b. */
static double orient(opt a, opt b, opt p) { return cross2(sub2(b, a), sub2(p, a)); }

/* Shoelace area of an ordered point list (paper Sec. II-B, `area`). */
static double shoelace(const opt* v, int n)
{
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += cross2(v[k], v[(k + 1) % n]);
    return 0.5 * s;
}

/* Crossing parameters of segment a->b with segment c->d.
 * r = b - a, s = d - c, q = c - a, D = cross(r, s),
 * a + t r = c + u s  =>  t = cross(q, s) / D, u = cross(q, r) / D. */
static int edge_cross(opt a, opt b, opt c, opt d, double* t, double* u, double* D)
{
    opt r = sub2(b, a), s = sub2(d, c), q = sub2(c, a);
    *D = cross2(r, s);
    if (*D == 0.0) return 0;
    *t = cross2(q, s) / *D;
    *u = cross2(q, r) / *D;
    return (*t > 0.0 && *t < 1.0 && *u > 0.0 && *u < 1.0);
}

static int bbox_overlap(opt a, opt b, opt c, opt d)
{
    double ax0 = fmin(a.x, b.x), ax1 = fmax(a.x, b.x), ay0 = fmin(a.y, b.y), ay1 = fmax(a.y, b.y);
    double cx0 = fmin(c.x, d.x), cx1 = fmax(c.x, d.x), cy0 = fmin(c.y, d.y), cy1 = fmax(c.y, d.y);
    return ax0 <= cx1 && cx0 <= ax1 && ay0 <= cy1 && cy0 <= ay1;
}

/* Near-degenerate classifier.  L is the largest |coordinate| of either
 * polygon in the frame whose origin is P1's vertex 0.  A pair is flagged when
 *   (i)   some vertex-vs-edge orientation has |orient| <= 1e-5 L^2, or
 *   (ii)  some proper crossing has t or u within 1e-5 of 0 or 1, or
 *   (iii) some pair of edges with overlapping bounding boxes has
 *         |cross(r, s)| <= 1e-5 |r| |s|. */
static int classify_degenerate(const opt* P, int n1, const opt* Q, int n2)
{
    opt o = P[0];
    double L = 0.0;
    for (int i = 0; i < n1; ++i) { L = fmax(L, fabs(P[i].x - o.x)); L = fmax(L, fabs(P[i].y - o.y)); }
    for (int j = 0; j < n2; ++j) { L = fmax(L, fabs(Q[j].x - o.x)); L = fmax(L, fabs(Q[j].y - o.y)); }
    if (L == 0.0) return 1;
    double thr = ORC_DEGEN_REL * L * L;
    for (int i = 0; i < n1; ++i) {
        opt a = P[i], b = P[(i + 1) % n1];
        for (int j = 0; j < n2; ++j) {
            opt c = Q[j], d = Q[(j + 1) % n2];
            if (fabs(orient(c, d, a)) <= thr) return 1;
            if (fabs(orient(a, b, c)) <= thr) return 1;
            double t, u, D;
            if (edge_cross(a, b, c, d, &t, &u, &D)) {
                if (t <= ORC_DEGEN_REL || t >= 1.0 - ORC_DEGEN_REL) return 1;
                if (u <= ORC_DEGEN_REL || u >= 1.0 - ORC_DEGEN_REL) return 1;
            }
            opt r = sub2(b, a), s = sub2(d, c);
            double nr = sqrt(r.x * r.x + r.y * r.y), ns = sqrt(s.x * s.x + s.y * s.y);
            if (fabs(cross2(r, s)) <= ORC_DEGEN_REL * nr * ns && bbox_overlap(a, b, c, d)) return 1;
        }
    }
    return 0;
}

static int inside_or_on(opt p, const opt* poly, int n)
{
    for (int j = 0; j < n; ++j)
        if (orient(poly[j], poly[(j + 1) % n], p) < 0.0) return 0;
    return 1;
}

/* Forward on one pair of double polygons (paper Sec. II-B `iou`). */
static void forward_pair(const opt* P, int n1, const opt* Q, int n2, int K, ofwd* out)
{
    int C = 2 * K;
    memset(out, 0, sizeof(*out));
    memset(out->code, 0xFF, sizeof(out->code));
    if (n1 < 3 || n1 > K || n2 < 3 || n2 > K) {
        out->status = ORC_ST_BAD_COUNT;
        return;
    }
    out->a1 = shoelace(P, n1);
    out->a2 = shoelace(Q, n2);
    out->degen = classify_degenerate(P, n1, Q, n2);

    ocand cand[ORC_MAXCAND];
    int m = 0;
    /* P1 vertices inside-or-on P2. */
    for (int i = 0; i < n1; ++i)
        if (inside_or_on(P[i], Q, n2)) { cand[m].p = P[i]; cand[m].code = (uint8_t)i; ++m; }
    /* P2 vertices inside-or-on P1, minus exact duplicates of P1 vertices. */
    for (int j = 0; j < n2; ++j) {
        int dup = 0;
        for (int i = 0; i < n1; ++i)
            if (Q[j].x == P[i].x && Q[j].y == P[i].y) dup = 1;
        if (!dup && inside_or_on(Q[j], P, n1)) { cand[m].p = Q[j]; cand[m].code = (uint8_t)(0x40 | j); ++m; }
    }
    /* Proper edge crossings. */
    for (int i = 0; i < n1; ++i) {
        opt a = P[i], b = P[(i + 1) % n1];
        for (int j = 0; j < n2; ++j) {
            double t, u, D;
            if (edge_cross(a, b, Q[j], Q[(j + 1) % n2], &t, &u, &D)) {
                opt x = {a.x + t * (b.x - a.x), a.y + t * (b.y - a.y)};
                cand[m].p = x;
                cand[m].code = (uint8_t)(0x80 | (i << 3) | j);
                ++m;
            }
        }
    }
    if (m > C) {
        out->status = ORC_ST_OVERFLOW;
        out->degen = 1;
        return;
    }
    if (m < 3) return; /* empty: nx = 0, IoU = 0 */

    /* Counter-clockwise order: sort by angle about the centroid (ties by code). */
    double cx = 0.0, cy = 0.0;
    for (int k = 0; k < m; ++k) { cx += cand[k].p.x; cy += cand[k].p.y; }
    cx /= m;
    cy /= m;
    for (int k = 0; k < m; ++k) cand[k].ang = atan2(cand[k].p.y - cy, cand[k].p.x - cx);
    for (int k = 1; k < m; ++k) {
        ocand v = cand[k];
        int l = k - 1;
        while (l >= 0 && (cand[l].ang > v.ang || (cand[l].ang == v.ang && cand[l].code > v.code))) {
            cand[l + 1] = cand[l];
            --l;
        }
        cand[l + 1] = v;
    }
    /* Rotate so that the smallest code is first. */
    int s0 = 0;
    for (int k = 1; k < m; ++k)
        if (cand[k].code < cand[s0].code) s0 = k;
    for (int k = 0; k < m; ++k) {
        out->code[k] = cand[(s0 + k) % m].code;
        out->w[k] = cand[(s0 + k) % m].p;
    }
    out->nx = m;
    out->ai = shoelace(out->w, m);
    double U = out->a1 + out->a2 - out->ai;
    out->iou = (U > 0.0) ? out->ai / U : 0.0;
}

/* Point named by a code (the backward's reconstruction from saved flags). */
static int point_of_code(uint8_t code, const opt* P, int n1, const opt* Q, int n2, opt* w)
{
    int kind = code >> 6;
    if (kind == 0) {
        int i = code & 0x3F;
        if (i >= n1) return 0;
        *w = P[i];
        return 1;
    }
    if (kind == 1) {
        int j = code & 0x3F;
        if (j >= n2) return 0;
        *w = Q[j];
        return 1;
    }
    if (kind == 2) {
        int i = (code >> 3) & 7, j = code & 7;
        if (i >= n1 || j >= n2) return 0;
        opt a = P[i], b = P[(i + 1) % n1], c = Q[j], d = Q[(j + 1) % n2];
        opt r = sub2(b, a), s = sub2(d, c), q = sub2(c, a);
        double D = cross2(r, s);
        if (D == 0.0) return 0;
        double t = cross2(q, s) / D;
        w->x = a.x + t * r.x;
        w->y = a.y + t * r.y;
        return 1;
    }
    return 0;
}

/* Area adjoint on one pair (paper Sec. II-B `iou_grad`, the part below the
 * IoU): given dL/dA_i (gai) and dL/dA_1, dL/dA_2 (ga1, ga2), the gradients of
 * L with respect to both polygons' vertices through the recorded (nx, codes).
 * Gradients are overwritten. */
static int area_backward_pair(const opt* P, int n1, const opt* Q, int n2, double gai, double ga1, double ga2, int nx,
                              const uint8_t* code, opt* g1, opt* g2)
{
    for (int i = 0; i < ORC_MAXK; ++i) { g1[i].x = g1[i].y = 0.0; g2[i].x = g2[i].y = 0.0; }
    if (n1 < 3 || n2 < 3) return ORC_ST_BAD_COUNT;
    opt w[ORC_MAXC];
    if (nx >= 3)
        for (int k = 0; k < nx; ++k)
            if (!point_of_code(code[k], P, n1, Q, n2, &w[k])) return ORC_ST_OVERFLOW;
    if (nx < 3) nx = 0; /* no intersection polygon: only the input areas */

    /* Shoelace adjoint: dA/dw_k = 1/2 (y_{k+1} - y_{k-1}, x_{k-1} - x_{k+1}). */
    for (int k = 0; k < nx; ++k) {
        opt wp = w[(k + nx - 1) % nx], wn = w[(k + 1) % nx];
        opt gw = {0.5 * gai * (wn.y - wp.y), 0.5 * gai * (wp.x - wn.x)};
        uint8_t c = code[k];
        int kind = c >> 6;
        if (kind == 0) {
            g1[c & 0x3F].x += gw.x;
            g1[c & 0x3F].y += gw.y;
        } else if (kind == 1) {
            g2[c & 0x3F].x += gw.x;
            g2[c & 0x3F].y += gw.y;
        } else {
            int i = (c >> 3) & 7, j = c & 7, i1 = (i + 1) % n1, j1 = (j + 1) % n2;
            opt a = P[i], b = P[i1], cc = Q[j], d = Q[j1];
            opt r = sub2(b, a), s = sub2(d, cc), q = sub2(cc, a);
            double N = cross2(q, s), D = cross2(r, s), t = N / D;
            /* P = a + t r */
            double gt = gw.x * r.x + gw.y * r.y;
            opt gr = {t * gw.x, t * gw.y};
            opt ga = gw;
            /* t = N / D */
            double gN = gt / D, gD = -gt * t / D;
            /* N = cross(q, s), D = cross(r, s) */
            opt gq = {gN * s.y, -gN * s.x};
            opt gs = {gN * (-q.y) + gD * (-r.y), gN * q.x + gD * r.x};
            gr.x += gD * s.y;
            gr.y += -gD * s.x;
            /* q = c - a, r = b - a, s = d - c */
            ga.x -= gq.x + gr.x;
            ga.y -= gq.y + gr.y;
            g1[i].x += ga.x;
            g1[i].y += ga.y;
            g1[i1].x += gr.x;
            g1[i1].y += gr.y;
            g2[j].x += gq.x - gs.x;
            g2[j].y += gq.y - gs.y;
            g2[j1].x += gs.x;
            g2[j1].y += gs.y;
        }
    }
    /* Areas of the inputs: same shoelace adjoint on P1 and P2. */
    for (int i = 0; i < n1; ++i) {
        opt pp = P[(i + n1 - 1) % n1], pn = P[(i + 1) % n1];
        g1[i].x += 0.5 * ga1 * (pn.y - pp.y);
        g1[i].y += 0.5 * ga1 * (pp.x - pn.x);
    }
    for (int j = 0; j < n2; ++j) {
        opt qp = Q[(j + n2 - 1) % n2], qn = Q[(j + 1) % n2];
        g2[j].x += 0.5 * ga2 * (qn.y - qp.y);
        g2[j].y += 0.5 * ga2 * (qp.x - qn.x);
    }
    return 0;
}

/* Backward on one pair: dL/dIoU -> dL/dP1, dL/dP2.  IoU = ai / U with
 * U = a1 + a2 - ai, so dIoU/dai = (a1 + a2) / U^2 and dIoU/da1 = dIoU/da2 =
 * -ai / U^2; nx < 3 or U <= 0 give zero gradients. */
static int backward_pair(const opt* P, int n1, const opt* Q, int n2, double g, int nx, const uint8_t* code,
                         opt* g1, opt* g2)
{
    for (int i = 0; i < ORC_MAXK; ++i) { g1[i].x = g1[i].y = 0.0; g2[i].x = g2[i].y = 0.0; }
    if (n1 < 3 || n2 < 3) return ORC_ST_BAD_COUNT;
    if (nx < 3) return 0;
    opt w[ORC_MAXC];
    for (int k = 0; k < nx; ++k)
        if (!point_of_code(code[k], P, n1, Q, n2, &w[k])) return ORC_ST_OVERFLOW;
    double a1 = shoelace(P, n1), a2 = shoelace(Q, n2), ai = shoelace(w, nx);
    double U = a1 + a2 - ai;
    if (!(U > 0.0)) return 0;
    double gai = g * (a1 + a2) / (U * U);
    double ga12 = -g * ai / (U * U);
    return area_backward_pair(P, n1, Q, n2, gai, ga12, ga12, nx, code, g1, g2);
}

static int load_f32(const float* src, int n, opt* dst)
{
    for (int v = 0; v < n; ++v) { dst[v].x = (double)src[2 * v]; dst[v].y = (double)src[2 * v + 1]; }
    return n;
}

static int count_of(const uint8_t* c, int64_t k, int K) { return c ? (int)c[k] : K; }

/* ---------------------------------------------------------------- exports */

/* Batch forward on FP32 polygons [n][K][2] (promoted exactly to double).
 * counts may be NULL (all K).  xflags is [n][2K].  Returns OR of status bits. */
int oracle_iou_paired(int64_t n, int K, const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2,
                      double* iou, uint8_t* nx, uint8_t* xflags, uint8_t* degen, double* areas /* [n][3] or NULL */)
{
    if (K < 3 || K > ORC_MAXK) return -1;
    int st = 0;
    for (int64_t k = 0; k < n; ++k) {
        opt P[ORC_MAXK], Q[ORC_MAXK];
        int n1 = count_of(c1, k, K), n2 = count_of(c2, k, K);
        ofwd f;
        if (n1 < 3 || n1 > K || n2 < 3 || n2 > K) {
            memset(&f, 0, sizeof(f));
            memset(f.code, 0xFF, sizeof(f.code));
            f.status = ORC_ST_BAD_COUNT;
        } else {
            load_f32(p1 + k * 2 * K, n1, P);
            load_f32(p2 + k * 2 * K, n2, Q);
            forward_pair(P, n1, Q, n2, K, &f);
        }
        st |= f.status;
        iou[k] = f.iou;
        if (nx) nx[k] = (uint8_t)f.nx;
        if (xflags) memcpy(xflags + k * 2 * K, f.code, (size_t)(2 * K));
        if (degen) degen[k] = (uint8_t)f.degen;
        if (areas) { areas[3 * k] = f.ai; areas[3 * k + 1] = f.a1; areas[3 * k + 2] = f.a2; }
    }
    return st;
}

/* Batch `intersect` (paper Sec. II-B: intersect(p1, p2, xflags) returns the
 * intersection polygon with its vertex count): verts [n][2K][2] receives the
 * vertices in the order of xflags (counter-clockwise from the smallest code),
 * unused slots 0; nx, xflags as oracle_iou_paired.  Returns OR of status
 * bits. */
int oracle_intersect_paired(int64_t n, int K, const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2,
                            double* verts, uint8_t* nx, uint8_t* xflags)
{
    if (K < 3 || K > ORC_MAXK) return -1;
    int st = 0;
    for (int64_t k = 0; k < n; ++k) {
        opt P[ORC_MAXK], Q[ORC_MAXK];
        int n1 = count_of(c1, k, K), n2 = count_of(c2, k, K);
        ofwd f;
        memset(&f, 0, sizeof(f));
        memset(f.code, 0xFF, sizeof(f.code));
        if (n1 < 3 || n1 > K || n2 < 3 || n2 > K) {
            f.status = ORC_ST_BAD_COUNT;
        } else {
            load_f32(p1 + k * 2 * K, n1, P);
            load_f32(p2 + k * 2 * K, n2, Q);
            forward_pair(P, n1, Q, n2, K, &f);
        }
        st |= f.status;
        for (int v = 0; v < 2 * K; ++v) {
            verts[(k * 2 * K + v) * 2] = v < f.nx ? f.w[v].x : 0.0;
            verts[(k * 2 * K + v) * 2 + 1] = v < f.nx ? f.w[v].y : 0.0;
        }
        if (nx) nx[k] = (uint8_t)f.nx;
        if (xflags) memcpy(xflags + k * 2 * K, f.code, (size_t)(2 * K));
    }
    return st;
}

/* Batch `area` (paper Sec. II-B listing: area(p) of a polygon): the shoelace
 * area of each polygon [n][K][2] with its count (NULL: K); 0 for a count
 * outside [3, K]. */
int oracle_area(int64_t n, int K, const float* p, const uint8_t* c, double* area)
{
    if (K < 3 || K > ORC_MAXK) return -1;
    int st = 0;
    for (int64_t k = 0; k < n; ++k) {
        opt P[ORC_MAXK];
        int m = count_of(c, k, K);
        if (m < 3 || m > K) {
            area[k] = 0.0;
            st |= ORC_ST_BAD_COUNT;
            continue;
        }
        load_f32(p + k * 2 * K, m, P);
        area[k] = shoelace(P, m);
    }
    return st;
}

/* Batch backward: grad [n], (nx, xflags) as recorded, grads [n][K][2] double. */
int oracle_iou_backward_paired(int64_t n, int K, const float* p1, const uint8_t* c1, const float* p2,
                               const uint8_t* c2, const double* grad, const uint8_t* nx, const uint8_t* xflags,
                               double* g1, double* g2)
{
    if (K < 3 || K > ORC_MAXK) return -1;
    int st = 0;
    for (int64_t k = 0; k < n; ++k) {
        opt P[ORC_MAXK], Q[ORC_MAXK], G1[ORC_MAXK], G2[ORC_MAXK];
        int n1 = count_of(c1, k, K), n2 = count_of(c2, k, K);
        memset(G1, 0, sizeof(G1));
        memset(G2, 0, sizeof(G2));
        if (n1 < 3 || n1 > K || n2 < 3 || n2 > K) {
            st |= ORC_ST_BAD_COUNT;
        } else {
            load_f32(p1 + k * 2 * K, n1, P);
            load_f32(p2 + k * 2 * K, n2, Q);
            st |= backward_pair(P, n1, Q, n2, grad[k], nx[k], xflags + k * 2 * K, G1, G2);
        }
        for (int v = 0; v < K; ++v) {
            g1[(k * K + v) * 2] = G1[v].x;
            g1[(k * K + v) * 2 + 1] = G1[v].y;
            g2[(k * K + v) * 2] = G2[v].x;
            g2[(k * K + v) * 2 + 1] = G2[v].y;
        }
    }
    return st;
}

/* Batch area adjoint: dL/dA_i, dL/dA_1, dL/dA_2 per pair [n] -> grads
 * [n][K][2] double through the recorded (nx, xflags). */
int oracle_area_backward_paired(int64_t n, int K, const float* p1, const uint8_t* c1, const float* p2,
                                const uint8_t* c2, const double* gai, const double* ga1, const double* ga2,
                                const uint8_t* nx, const uint8_t* xflags, double* g1, double* g2)
{
    if (K < 3 || K > ORC_MAXK) return -1;
    int st = 0;
    for (int64_t k = 0; k < n; ++k) {
        opt P[ORC_MAXK], Q[ORC_MAXK], G1[ORC_MAXK], G2[ORC_MAXK];
        int n1 = count_of(c1, k, K), n2 = count_of(c2, k, K);
        memset(G1, 0, sizeof(G1));
        memset(G2, 0, sizeof(G2));
        if (n1 < 3 || n1 > K || n2 < 3 || n2 > K) {
            st |= ORC_ST_BAD_COUNT;
        } else {
            load_f32(p1 + k * 2 * K, n1, P);
            load_f32(p2 + k * 2 * K, n2, Q);
            st |= area_backward_pair(P, n1, Q, n2, gai[k], ga1[k], ga2[k], nx[k], xflags + k * 2 * K, G1, G2);
        }
        for (int v = 0; v < K; ++v) {
            g1[(k * K + v) * 2] = G1[v].x;
            g1[(k * K + v) * 2 + 1] = G1[v].y;
            g2[(k * K + v) * 2] = G2[v].x;
            g2[(k * K + v) * 2 + 1] = G2[v].y;
        }
    }
    return st;
}

/* N x M matrix of IoU and nx (row i = a[i], column j = b[j]). */
int oracle_iou_pairwise(int64_t N, int64_t M, int K, const float* a, const uint8_t* ca, const float* b,
                        const uint8_t* cb, double* iou, uint8_t* nx)
{
    if (K < 3 || K > ORC_MAXK) return -1;
    int st = 0;
    for (int64_t i = 0; i < N; ++i) {
        opt P[ORC_MAXK];
        int n1 = count_of(ca, i, K);
        if (n1 >= 3 && n1 <= K) load_f32(a + i * 2 * K, n1, P);
        for (int64_t j = 0; j < M; ++j) {
            opt Q[ORC_MAXK];
            int n2 = count_of(cb, j, K);
            ofwd f;
            if (n1 < 3 || n1 > K || n2 < 3 || n2 > K) {
                memset(&f, 0, sizeof(f));
                f.status = ORC_ST_BAD_COUNT;
            } else {
                load_f32(b + j * 2 * K, n2, Q);
                forward_pair(P, n1, Q, n2, K, &f);
            }
            st |= f.status;
            iou[i * M + j] = f.iou;
            if (nx) nx[i * M + j] = (uint8_t)f.nx;
        }
    }
    return st;
}

/* Double-precision single-pair forward (for finite differences).
 * out = {iou, ai, a1, a2}; code has 2K slots. */
int oracle_iou_pair_f64(int K, const double* p1, int n1, const double* p2, int n2, double* out, int* nx,
                        uint8_t* code, int* degen)
{
    if (K < 3 || K > ORC_MAXK) return -1;
    opt P[ORC_MAXK], Q[ORC_MAXK];
    for (int v = 0; v < n1 && v < ORC_MAXK; ++v) { P[v].x = p1[2 * v]; P[v].y = p1[2 * v + 1]; }
    for (int v = 0; v < n2 && v < ORC_MAXK; ++v) { Q[v].x = p2[2 * v]; Q[v].y = p2[2 * v + 1]; }
    ofwd f;
    forward_pair(P, n1, Q, n2, K, &f);
    out[0] = f.iou;
    out[1] = f.ai;
    out[2] = f.a1;
    out[3] = f.a2;
    *nx = f.nx;
    memcpy(code, f.code, (size_t)(2 * K));
    *degen = f.degen;
    return f.status;
}

/* Double-precision single-pair backward; g1, g2 are [K][2]. */
int oracle_iou_backward_pair_f64(int K, const double* p1, int n1, const double* p2, int n2, double grad, int nx,
                                 const uint8_t* code, double* g1, double* g2)
{
    if (K < 3 || K > ORC_MAXK) return -1;
    opt P[ORC_MAXK], Q[ORC_MAXK], G1[ORC_MAXK], G2[ORC_MAXK];
    for (int v = 0; v < n1 && v < ORC_MAXK; ++v) { P[v].x = p1[2 * v]; P[v].y = p1[2 * v + 1]; }
    for (int v = 0; v < n2 && v < ORC_MAXK; ++v) { Q[v].x = p2[2 * v]; Q[v].y = p2[2 * v + 1]; }
    int st = backward_pair(P, n1, Q, n2, grad, nx, code, G1, G2);
    for (int v = 0; v < K; ++v) {
        g1[2 * v] = G1[v].x;
        g1[2 * v + 1] = G1[v].y;
        g2[2 * v] = G2[v].x;
        g2[2 * v + 1] = G2[v].y;
    }
    return st;
}


/* ------------------------------------------- GIoU / DIoU terms of the loss
 *
 * The IoU-loss case study (paper Sec. IV-A) trains rotated boxes with
 * 1 - IoU.  Its generalized and distance-penalised variants (the paper names
 * the IoU loss only; these are the standard extensions) add, per pair:
 *   GIoU = IoU - (A_h - U) / A_h,  A_h = area of the convex hull of both
 *          polygons' vertices, U = A_1 + A_2 - A_i;
 *   DIoU = IoU - rho2 / c2,  rho2 = squared distance between the two
 *          polygons' vertex means, c2 = squared diameter of that hull (the
 *          largest squared distance between any two of the vertices).
 * The loss term of a pair is w (1 - GIoU) or w (1 - DIoU).  The hull is
 * Andrew's monotone chain over the n1 + n2 points in double (points sorted by
 * x, then y; collinear points dropped); its gradient is the shoelace adjoint
 * over the hull's vertices, each routed to the input vertex it came from.
 * The diameter takes the first largest pair in index order (P1's vertices,
 * then P2's), and its gradient goes to that pair. */

typedef struct {
    opt p;
    int src; /* 0..n1-1: P1 vertex, n1..: P2 vertex */
} hpt;

/* Convex hull (counter-clockwise, no collinear points) of m points; returns
 * the number of hull vertices written to hull[]. */
static int monotone_chain(hpt* pts, int m, hpt* hull)
{
    for (int k = 1; k < m; ++k) {
        hpt v = pts[k];
        int l = k - 1;
        while (l >= 0 && (pts[l].p.x > v.p.x || (pts[l].p.x == v.p.x && pts[l].p.y > v.p.y))) {
            pts[l + 1] = pts[l];
            --l;
        }
        pts[l + 1] = v;
    }
    int h = 0;
    for (int k = 0; k < m; ++k) { /* lower chain */
        while (h >= 2 && orient(hull[h - 2].p, hull[h - 1].p, pts[k].p) <= 0.0) --h;
        hull[h++] = pts[k];
    }
    for (int k = m - 2, lo = h + 1; k >= 0; --k) { /* upper chain */
        while (h >= lo && orient(hull[h - 2].p, hull[h - 1].p, pts[k].p) <= 0.0) --h;
        hull[h++] = pts[k];
    }
    return h > 1 ? h - 1 : h; /* the last point repeats the first */
}

typedef struct {
    double ah, rho2, c2;
    int h;
    hpt hull[4 * ORC_MAXK + 1]; /* the chains hold up to 2 m points while they are built */
    int da, db; /* the diameter's pair (indices into P1 ++ P2) */
} ohull;

static void hull_terms(const opt* P, int n1, const opt* Q, int n2, ohull* o)
{
    hpt pts[2 * ORC_MAXK];
    int m = 0;
    for (int i = 0; i < n1; ++i) { pts[m].p = P[i]; pts[m].src = i; ++m; }
    for (int j = 0; j < n2; ++j) { pts[m].p = Q[j]; pts[m].src = n1 + j; ++m; }
    o->h = monotone_chain(pts, m, o->hull);
    opt hv[4 * ORC_MAXK];
    for (int k = 0; k < o->h; ++k) hv[k] = o->hull[k].p;
    o->ah = o->h >= 3 ? shoelace(hv, o->h) : 0.0;
    opt m1 = {0.0, 0.0}, m2 = {0.0, 0.0};
    for (int i = 0; i < n1; ++i) { m1.x += P[i].x; m1.y += P[i].y; }
    for (int j = 0; j < n2; ++j) { m2.x += Q[j].x; m2.y += Q[j].y; }
    m1.x /= n1; m1.y /= n1; m2.x /= n2; m2.y /= n2;
    o->rho2 = (m1.x - m2.x) * (m1.x - m2.x) + (m1.y - m2.y) * (m1.y - m2.y);
    opt all[2 * ORC_MAXK];
    for (int i = 0; i < n1; ++i) all[i] = P[i];
    for (int j = 0; j < n2; ++j) all[n1 + j] = Q[j];
    o->c2 = -1.0;
    o->da = o->db = 0;
    for (int a = 0; a < n1 + n2; ++a)
        for (int b = a + 1; b < n1 + n2; ++b) {
            double d = (all[a].x - all[b].x) * (all[a].x - all[b].x) + (all[a].y - all[b].y) * (all[a].y - all[b].y);
            if (d > o->c2) { o->c2 = d; o->da = a; o->db = b; }
        }
}

static void add_to(opt* g1, opt* g2, int n1, int src, double gx, double gy)
{
    if (src < n1) { g1[src].x += gx; g1[src].y += gy; }
    else { g2[src - n1].x += gx; g2[src - n1].y += gy; }
}

/* Loss term and its gradient on one pair (variant 1: GIoU, 2: DIoU):
 * *lk = w (1 - GIoU) or w (1 - DIoU); g1, g2 = d lk / d P, d Q.
 * Zero (and *lk = w) for U <= 0 or a degenerate hull / diameter. */
static int loss_variant_pair(const opt* P, int n1, const opt* Q, int n2, int K, int variant, double w, double* lk,
                             double* terms, opt* g1, opt* g2)
{
    ofwd f;
    forward_pair(P, n1, Q, n2, K, &f);
    ohull hq;
    hull_terms(P, n1, Q, n2, &hq);
    double U = f.a1 + f.a2 - f.ai;
    double iou = f.iou;
    terms[0] = iou;
    terms[1] = hq.ah;
    terms[2] = hq.rho2;
    terms[3] = hq.c2;
    for (int i = 0; i < ORC_MAXK; ++i) { g1[i].x = g1[i].y = 0.0; g2[i].x = g2[i].y = 0.0; }
    if (!(U > 0.0)) { *lk = w; return f.status; }
    int nx = f.nx >= 3 ? f.nx : 0;
    /* d IoU / d(A_i, A_1, A_2) (zero without an intersection polygon) */
    double di = nx ? (f.a1 + f.a2) / (U * U) : 0.0, d12 = nx ? -f.ai / (U * U) : 0.0;
    double gai, ga1, ga2;
    if (variant == 1) {
        if (!(hq.ah > 0.0)) { *lk = w * (1.0 - iou); return f.status; }
        *lk = w * (1.0 - iou + (hq.ah - U) / hq.ah);
        /* lk = w (2 - IoU - U / A_h) */
        gai = w * (-di + 1.0 / hq.ah);
        ga1 = ga2 = w * (-d12 - 1.0 / hq.ah);
    } else {
        if (!(hq.c2 > 0.0)) { *lk = w * (1.0 - iou); return f.status; }
        *lk = w * (1.0 - iou + hq.rho2 / hq.c2);
        gai = -w * di;
        ga1 = ga2 = -w * d12;
    }
    int st = area_backward_pair(P, n1, Q, n2, gai, ga1, ga2, nx, f.code, g1, g2);
    if (variant == 1) {
        /* hull area: shoelace adjoint over the hull's vertices */
        double gh = w * U / (hq.ah * hq.ah);
        for (int k = 0; k < hq.h; ++k) {
            opt hp = hq.hull[(k + hq.h - 1) % hq.h].p, hn = hq.hull[(k + 1) % hq.h].p;
            add_to(g1, g2, n1, hq.hull[k].src, 0.5 * gh * (hn.y - hp.y), 0.5 * gh * (hp.x - hn.x));
        }
    } else {
        /* rho2 / c2 */
        opt m1 = {0.0, 0.0}, m2 = {0.0, 0.0};
        for (int i = 0; i < n1; ++i) { m1.x += P[i].x; m1.y += P[i].y; }
        for (int j = 0; j < n2; ++j) { m2.x += Q[j].x; m2.y += Q[j].y; }
        m1.x /= n1; m1.y /= n1; m2.x /= n2; m2.y /= n2;
        double gr = w / hq.c2, gc = -w * hq.rho2 / (hq.c2 * hq.c2);
        for (int i = 0; i < n1; ++i) { g1[i].x += gr * 2.0 * (m1.x - m2.x) / n1; g1[i].y += gr * 2.0 * (m1.y - m2.y) / n1; }
        for (int j = 0; j < n2; ++j) { g2[j].x -= gr * 2.0 * (m1.x - m2.x) / n2; g2[j].y -= gr * 2.0 * (m1.y - m2.y) / n2; }
        opt pa = hq.da < n1 ? P[hq.da] : Q[hq.da - n1], pb = hq.db < n1 ? P[hq.db] : Q[hq.db - n1];
        add_to(g1, g2, n1, hq.da, gc * 2.0 * (pa.x - pb.x), gc * 2.0 * (pa.y - pb.y));
        add_to(g1, g2, n1, hq.db, -gc * 2.0 * (pa.x - pb.x), -gc * 2.0 * (pa.y - pb.y));
    }
    return f.status | st;
}

/* Batch loss terms of the GIoU (variant 1) or DIoU (variant 2) loss:
 * lk [n] = w_k (1 - GIoU_k) or w_k (1 - DIoU_k) (w = NULL: 1); terms [n][4] =
 * (IoU, A_h, rho2, c2) or NULL; g1, g2 [n][K][2] = d lk / d p1, d p2 (or
 * NULL).  Returns OR of status bits. */
int oracle_loss_variant_paired(int64_t n, int K, const float* p1, const uint8_t* c1, const float* p2,
                               const uint8_t* c2, int variant, const double* w, double* lk, double* terms, double* g1,
                               double* g2)
{
    if (K < 3 || K > ORC_MAXK || (variant != 1 && variant != 2)) return -1;
    int st = 0;
    for (int64_t k = 0; k < n; ++k) {
        opt P[ORC_MAXK], Q[ORC_MAXK], G1[ORC_MAXK], G2[ORC_MAXK];
        double tm[4] = {0.0, 0.0, 0.0, 0.0};
        int n1 = count_of(c1, k, K), n2 = count_of(c2, k, K);
        double wk = w ? w[k] : 1.0;
        memset(G1, 0, sizeof(G1));
        memset(G2, 0, sizeof(G2));
        if (n1 < 3 || n1 > K || n2 < 3 || n2 > K) {
            st |= ORC_ST_BAD_COUNT;
            lk[k] = wk;
        } else {
            load_f32(p1 + k * 2 * K, n1, P);
            load_f32(p2 + k * 2 * K, n2, Q);
            st |= loss_variant_pair(P, n1, Q, n2, K, variant, wk, &lk[k], tm, G1, G2);
        }
        if (terms) memcpy(terms + 4 * k, tm, sizeof(tm));
        for (int v = 0; v < K; ++v) {
            if (g1) { g1[(k * K + v) * 2] = G1[v].x; g1[(k * K + v) * 2 + 1] = G1[v].y; }
            if (g2) { g2[(k * K + v) * 2] = G2[v].x; g2[(k * K + v) * 2 + 1] = G2[v].y; }
        }
    }
    return st;
}

/* Double-precision single-pair loss term (for finite differences). */
int oracle_loss_variant_pair_f64(int K, const double* p1, int n1, const double* p2, int n2, int variant, double w,
                                 double* lk, double* g1, double* g2)
{
    if (K < 3 || K > ORC_MAXK || (variant != 1 && variant != 2)) return -1;
    opt P[ORC_MAXK], Q[ORC_MAXK], G1[ORC_MAXK], G2[ORC_MAXK];
    for (int v = 0; v < n1 && v < ORC_MAXK; ++v) { P[v].x = p1[2 * v]; P[v].y = p1[2 * v + 1]; }
    for (int v = 0; v < n2 && v < ORC_MAXK; ++v) { Q[v].x = p2[2 * v]; Q[v].y = p2[2 * v + 1]; }
    double tm[4];
    int st = loss_variant_pair(P, n1, Q, n2, K, variant, w, lk, tm, G1, G2);
    for (int v = 0; v < K; ++v) {
        if (g1) { g1[2 * v] = G1[v].x; g1[2 * v + 1] = G1[v].y; }
        if (g2) { g2[2 * v] = G2[v].x; g2[2 * v + 1] = G2[v].y; }
    }
    return st;
}
