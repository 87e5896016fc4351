// K = 8 paired kernels: a group of 8 lanes per pair (4 pairs per warp).
//
// With K = 8 a thread-per-pair kernel unrolls 64 vertex-edge blocks and its
// code no longer fits the instruction cache.  Here lane r of a group owns
// P1's vertex r and edge r (r < n1) and P2's edge r (r < n2), and keeps a copy
// of P2; every per-lane loop runs over 8, so the code stays small.  All
// shuffles use the group's own lane mask, and every branch that leads to a
// shuffle depends only on group-wide values, so groups of a warp may diverge.
//
// Forward (paper Sec. II-B `iou`): lane r computes row r of the orientation
// tables, S(r,j) = orient(b_j, b_j+1, a_r) and T(r,j) = orient(a_r, a_r+1, b_j);
// the rows are OR-combined into 64-bit sign masks, after which every lane
// knows the inside vertices and the crossings (as in fwd_generic); with
// refinement, orientations under the routing threshold first take the FP64
// definition's sign in their own lane's row (refine_row8).  The area
// is fwd_generic's select-free sum: lane r adds P1 edge r's vertex term and
// its row of crossing terms, a group sum adds them up.  Lane r also builds
// its chunk of the counter-clockwise vertex order: vertex r if inside, the
// entry crossing of edge r, its exit crossing and the chain of P2 vertices
// that follows an exit.  An exclusive scan of chunk lengths places
// the chunks; the cycle is rotated to its smallest code.
//
// Backward (paper Sec. II-B `iou_grad`): the shape derivative over the
// clipped pieces (see bwd_shape).  Lane r evaluates P1 edge r and P2 edge r;
// the contribution of an edge to its end vertex moves to the next lane with
// one shuffle, and lane r stores vertex r's gradients.
#pragma once

#include "dgal_geom.cuh"

namespace dgal {
namespace g8 {

constexpr int G = 8;

__device__ __forceinline__ unsigned gmask() { return 0xFFu << ((threadIdx.x & 31) & ~7); }
__device__ __forceinline__ int gbase() { return (threadIdx.x & 31) & ~7; }

__device__ __forceinline__ uint64_t gor64(unsigned m, uint64_t v) {
#pragma unroll
    for (int off = 1; off < G; off <<= 1) v |= __shfl_xor_sync(m, v, off, G);
    return v;
}
__device__ __forceinline__ uint32_t gor32(unsigned m, uint32_t v) {
#pragma unroll
    for (int off = 1; off < G; off <<= 1) v |= __shfl_xor_sync(m, v, off, G);
    return v;
}
__device__ __forceinline__ float gsum(unsigned m, float v) {
#pragma unroll
    for (int off = 1; off < G; off <<= 1) v += __shfl_xor_sync(m, v, off, G);
    return v;
}
__device__ __forceinline__ float gmax(unsigned m, float v) {
#pragma unroll
    for (int off = 1; off < G; off <<= 1) v = fmaxf(v, __shfl_xor_sync(m, v, off, G));
    return v;
}
__device__ __forceinline__ float gmin(unsigned m, float v) {
#pragma unroll
    for (int off = 1; off < G; off <<= 1) v = fminf(v, __shfl_xor_sync(m, v, off, G));
    return v;
}

// Lane view of a pair: own P1 vertex / edge, all of P2, in P1's local frame.
struct Lane {
    float ax, ay, eax, eay;
    float bx[8], by[8], ebx[8], eby[8];
    float bxr, byr, ebxr, ebyr; // the lane's own P2 vertex r and edge r (= bx[r], ..., loaded directly)
    int n1, n2, r;
};

// KIN: the capacity of the stored polygons (8, or 4 for quadrilaterals taken
// by groups of 8 lanes; then lanes 4..7 hold padding and stay idle).
template <int KIN = 8>
__device__ __forceinline__ void load_lane(const float* __restrict__ p1, const float* __restrict__ p2, int n1, int n2,
                                          int r, Lane& L) {
    const float ox = __ldg(p1), oy = __ldg(p1 + 1);
    const int rr = (r < n1) ? r : 0;
    const int rn = (rr + 1 < n1) ? rr + 1 : 0;
    const float2 v = __ldg(reinterpret_cast<const float2*>(p1) + rr);
    const float2 w = __ldg(reinterpret_cast<const float2*>(p1) + rn);
    L.ax = v.x - ox;
    L.ay = v.y - oy;
    L.eax = (w.x - ox) - L.ax;
    L.eay = (w.y - oy) - L.ay;
    float qx[8], qy[8];
    if constexpr (KIN == 8) {
        load_poly<8>(p2, qx, qy);
    } else {
        float ux[KIN], uy[KIN];
        load_poly<KIN>(p2, ux, uy);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            qx[j] = ux[j < KIN ? j : 0];
            qy[j] = uy[j < KIN ? j : 0];
        }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        L.bx[j] = qx[j] - ox;
        L.by[j] = qy[j] - oy;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const bool wrap = j + 1 >= n2;
        L.ebx[j] = (wrap ? L.bx[0] : L.bx[(j + 1) & 7]) - L.bx[j];
        L.eby[j] = (wrap ? L.by[0] : L.by[(j + 1) & 7]) - L.by[j];
    }
    {
        // the lane's own P2 vertex and edge, with the arithmetic of the loop
        // above (so the values equal bx[r], by[r], ebx[r], eby[r])
        const int rr2 = (r < n2) ? r : 0;
        const int rn2 = (rr2 + 1 < n2) ? rr2 + 1 : 0;
        const float2 q0 = __ldg(reinterpret_cast<const float2*>(p2) + rr2);
        const float2 q1 = __ldg(reinterpret_cast<const float2*>(p2) + rn2);
        L.bxr = q0.x - ox;
        L.byr = q0.y - oy;
        L.ebxr = (q1.x - ox) - L.bxr;
        L.ebyr = (q1.y - oy) - L.byr;
    }
    L.n1 = n1;
    L.n2 = n2;
    L.r = r;
}

// The backward's lane view: only the lane's own P1 vertex / edge and P2
// vertex / edge; the other lanes' come by shuffle.  The values equal those of
// load_lane (same arithmetic).
struct LaneS {
    float ax, ay, eax, eay;
    float bxr, byr, ebxr, ebyr;
    int n1, n2, r;
};

template <int KIN = 8>
__device__ __forceinline__ void load_lane_slim(const float* __restrict__ p1, const float* __restrict__ p2, int n1,
                                               int n2, int r, LaneS& L) {
    const float ox = __ldg(p1), oy = __ldg(p1 + 1);
    const int rr = (r < n1) ? r : 0;
    const int rn = (rr + 1 < n1) ? rr + 1 : 0;
    const float2 v = __ldg(reinterpret_cast<const float2*>(p1) + rr);
    const float2 w = __ldg(reinterpret_cast<const float2*>(p1) + rn);
    L.ax = v.x - ox;
    L.ay = v.y - oy;
    L.eax = (w.x - ox) - L.ax;
    L.eay = (w.y - oy) - L.ay;
    const int rr2 = (r < n2) ? r : 0;
    const int rn2 = (rr2 + 1 < n2) ? rr2 + 1 : 0;
    const float2 q0 = __ldg(reinterpret_cast<const float2*>(p2) + rr2);
    const float2 q1 = __ldg(reinterpret_cast<const float2*>(p2) + rn2);
    L.bxr = q0.x - ox;
    L.byr = q0.y - oy;
    L.ebxr = (q1.x - ox) - L.bxr;
    L.ebyr = (q1.y - oy) - L.byr;
    L.n1 = n1;
    L.n2 = n2;
    L.r = r;
}

__device__ __forceinline__ uint64_t col0_mask() {
    uint64_t c = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) c |= 1ull << (8 * i);
    return c;
}

// FP64 sign repair of lane r's row (refinement on, r < n1): every orientation
// of the row within 3x the routing threshold thr takes the FP64 definition's
// sign (orient_raw, the definition's operand order, from the raw inputs).
// The row's FP32 values are formed again from the lane's data; the margin
// covers a different rounding (contraction) of that second evaluation.
// sneg, tneg: the row's FP32 sign bits (bit j: column j).  An exactly zero
// orientation (a vertex on the line of an edge) takes the sign it has when P2
// is translated by an infinitesimal (eps, eps^2) (tie_neg).  Returns the
// repaired bits (S in bits 0-7, T in bits 8-15) and the zero orientations
// (S in bits 16-23, T in bits 24-31), or bit 32 set when a zero sits on an
// edge of zero length.  It runs only for pairs with an orientation under the
// threshold.
__device__ __forceinline__ uint64_t refine_row8(const Lane& L, const float* __restrict__ raw1,
                                                const float* __restrict__ raw2, int n1, int n2, int r, float thr,
                                                uint32_t sneg, uint32_t tneg) {
    const float wide = 3.f * thr;
    const int rn = (r + 1 < n1) ? r + 1 : 0;
    uint32_t zs = 0, zt = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        if (j >= n2) break;
        const float dx = L.ax - L.bx[j], dy = L.ay - L.by[j];
        const float sv = L.ebx[j] * dy - L.eby[j] * dx;
        const float tv = L.eay * dx - L.eax * dy;
        if (!(fabsf(sv) > wide)) {
            const int j1 = (j + 1 < n2) ? j + 1 : 0;
            const double v = orient_raw(raw2, j, j1, raw1, r);
            uint32_t ng = (v < 0.0) ? 1u : 0u;
            if (v == 0.0) {
                ng = tie_neg(raw2, j, j1, false);
                if (ng > 1u) return 1ull << 32;
                zs |= 1u << j;
            }
            sneg = ng ? (sneg | (1u << j)) : (sneg & ~(1u << j));
        }
        if (!(fabsf(tv) > wide)) {
            const double v = orient_raw(raw1, r, rn, raw2, j);
            uint32_t ng = (v < 0.0) ? 1u : 0u;
            if (v == 0.0) {
                ng = tie_neg(raw1, r, rn, true);
                if (ng > 1u) return 1ull << 32;
                zt |= 1u << j;
            }
            tneg = ng ? (tneg | (1u << j)) : (tneg & ~(1u << j));
        }
    }
    return (uint64_t)((sneg & 0xFFu) | ((tneg & 0xFFu) << 8) | (zs << 16) | (zt << 24));
}

struct FwdG {
    uint64_t w0, w1; // the 16 code bytes
    float iou;
    uint32_t nx;
    uint32_t degen; // near-degenerate (some orientation within kDegenRel L^2)
    float ai, a1, a2;
};

// Group forward.  Returns false (in every lane of the group) when the pair
// must take the warp-cooperative robust path.  raw1, raw2 (refinement on):
// the pair's input polygons; orientations under the routing threshold then
// take the FP64 definition's sign (refine_row8), exact zeros the sign under
// an infinitesimal translation of P2, and only a zero-length edge hands the
// pair back.  Their FP32 values still place the crossing points, as in the
// quadrilateral forward.
template <int KIN = 8>
__device__ __forceinline__ bool fwd_group(const Lane& L, FwdG& out, const float* __restrict__ raw1 = nullptr,
                                          const float* __restrict__ raw2 = nullptr) {
    const unsigned gm = gmask();
    const int base = gbase();
    const int r = L.r, n1 = L.n1, n2 = L.n2;
    const bool liveA = r < n1, liveB = r < n2;
    // Identical polygons (bit-equal vertices in the same order): by the
    // candidate rules the intersection is P1 itself (every P1 vertex is on
    // P2's boundary, P2's vertices are exact duplicates and no crossing is
    // proper), so IoU = 1 and the codes are P1's vertices in order.  The pair
    // is near-degenerate (its orientations vanish) and needs no test at all.
    if (n1 == n2 && !gor32(gm, (liveA && (L.ax != L.bxr || L.ay != L.byr)) ? 1u : 0u)) {
        const float a = 0.5f * gsum(gm, liveA ? L.ax * L.eay - L.ay * L.eax : 0.f);
        const uint64_t seq = 0x0706050403020100ull;
        out.w0 = n1 >= 8 ? seq : (seq | (~0ull << (8 * n1)));
        out.w1 = ~0ull;
        out.nx = (uint32_t)n1;
        out.ai = out.a1 = out.a2 = a;
        out.iou = a > 0.f ? 1.f : 0.f;
        out.degen = 1u;
        return true;
    }
    // L: the largest |coordinate| over both polygons (lane r contributes its
    // own P1 and P2 vertex)
    const float Lr = gmax(gm, fmaxf(liveA ? fmaxf(fabsf(L.ax), fabsf(L.ay)) : 0.f,
                                    liveB ? fmaxf(fabsf(L.bxr), fabsf(L.byr)) : 0.f));
    const float thr = kRouteRel * Lr * Lr;

    // row r of S and T, and the row's crossing terms of the area (see below);
    // j runs downwards so that the funnel shifts leave the sign of column j
    // in bit j
    uint32_t sneg = 0, tneg = 0;
    float mn = __int_as_float(0x7f800000);
    float term[8];
#pragma unroll
    for (int j = 7; j >= 0; --j) {
        const float dx = L.ax - L.bx[j], dy = L.ay - L.by[j];
        const float s = L.ebx[j] * dy - L.eby[j] * dx;
        const float t = L.eay * dx - L.eax * dy;
        mn = fminf(mn, (liveA && j < n2) ? fminf(fabsf(s), fabsf(t)) : __int_as_float(0x7f800000));
        sneg = push_sign(sneg, s);
        tneg = push_sign(tneg, t);
        const float D = L.eax * L.eby[j] - L.eay * L.ebx[j];
        const float c = L.ax * L.by[j] - L.ay * L.bx[j];
        term[j] = fmaf(c, D, s * t) * __fdividef(1.0f, fabsf(D));
    }
    mn = gmin(gm, mn);
    if (!(Lr > 0.f)) return false;
    uint32_t refined = 0u, zrow = 0u;
    bool tie = false; // some orientation of the pair is exactly zero (group-uniform)
    if (!(mn > thr)) {
        if (raw1 == nullptr) return false;
        const uint64_t rr = liveA ? refine_row8(L, raw1, raw2, n1, n2, r, thr, sneg, tneg) : 0ull;
        const uint32_t gf = gor32(gm, (uint32_t)(rr >> 32) | ((((uint32_t)rr >> 16) != 0u) ? 2u : 0u));
        if (gf & 1u) return false;
        tie = (gf & 2u) != 0u;
        if (liveA) {
            sneg = (uint32_t)rr & 0xFFu;
            tneg = (uint32_t)(rr >> 8) & 0xFFu;
            zrow = (uint32_t)rr >> 16;
        }
        refined = 2u;
    }
    out.degen = ((mn <= kDegenRel * Lr * Lr) ? 1u : 0u) | refined;
    const uint32_t colv = (1u << n2) - 1u;
    const uint64_t col0 = 0x0101010101010101ull;
    const uint64_t rows = (n1 >= 8) ? ~0ull : ((1ull << (8 * n1)) - 1ull);
    const uint64_t cols = col0 * colv;
    const uint64_t V = rows & cols;
    uint64_t sp, tp, X, entry1, exit1;
    uint32_t in1, in2, cnt;
    for (int pass = 0;; ++pass) {
        sp = gor64(gm, liveA ? (uint64_t)(~sneg & colv) << (8 * r) : 0ull);
        tp = gor64(gm, liveA ? (uint64_t)(~tneg & colv) << (8 * r) : 0ull);
        const uint64_t sp_next = ((sp >> 8) & ~(0xFFull << (8 * (n1 - 1)))) | ((sp & 0xFFull) << (8 * (n1 - 1)));
        const uint64_t tp_next = ((tp >> 1) & ~(col0 << (n2 - 1))) | ((tp & col0) << (n2 - 1));
        X = (sp ^ sp_next) & (tp ^ tp_next) & V;
        entry1 = X & ~sp;
        exit1 = X & sp;
        if ((X & tp) != entry1) return false;
        // in1: rows of sp equal to all valid columns (exact zero-byte test on sp ^ cols)
        const uint64_t z = (sp ^ cols) & rows;
        const uint64_t hi7 = 0x7F7F7F7F7F7F7F7Full;
        const uint64_t zb = ~(((z & hi7) + hi7) | z | hi7) & rows; // 0x80 in each zero byte of a valid row
        in1 = (uint32_t)(((zb >> 7) * 0x0102040810204080ull) >> 56);
        // in2: columns of tp set in every valid row (AND over the rows' bytes)
        uint64_t a = tp | ~rows;
        a &= a >> 32;
        a &= a >> 16;
        a &= a >> 8;
        in2 = (uint32_t)(a & 0xFFull) & colv;
        cnt = (uint32_t)(__popc(in1) + __popc(in2) + __popcll(X));
        // A pair with an exactly zero orientation whose clip under the
        // translation by (eps, eps^2) is not empty is clipped once more under
        // the opposite translation (-eps, -eps^2), which flips the sign of every
        // zero: an equally valid perturbation with the same limit area.  When
        // the interiors do not meet (a shared edge, a touching vertex), the
        // directions that make them overlap form a cone narrower than a
        // half-plane, so one of the two translations separates the polygons,
        // and the pair gets an empty clip instead of a sliver of zero area.
        if (pass == 1 || !tie || cnt == 0u) break;
        sneg ^= zrow & 0xFFu;
        tneg ^= zrow >> 8;
    }
    out.nx = 0;
    out.iou = 0.f;
    out.ai = 0.f;
    out.w0 = out.w1 = ~0ull;
    // the inputs' areas (kept for the union also when the intersection is empty)
    const float c1r = L.ax * L.eay - L.ay * L.eax;
    const float c2r = L.bxr * L.ebyr - L.byr * L.ebxr;
    const float a1 = 0.5f * gsum(gm, liveA ? c1r : 0.f);
    const float a2 = 0.5f * gsum(gm, liveB ? c2r : 0.f);
    out.a1 = a1;
    out.a2 = a2;
    if (cnt == 0u) return true;
    if (cnt < 3u || cnt > 16u) return false;

    // Area (the select-free shoelace of fwd_generic): every inside vertex
    // a_i+1 adds cross(a_i, ea_i), every inside b_j+1 adds cross(b_j, eb_j),
    // and every proper crossing (i, j) adds (cross(a_i, b_j) D + S T) / |D|,
    // with one crossing point shared by its two pieces and an FP32 error of
    // order u L^2 at any crossing angle.  Lane r adds P1 edge r's vertex term
    // and its row of crossing terms, and P2 edge r's vertex term.
    const uint32_t rowE = liveA ? (uint32_t)((entry1 >> (8 * r)) & 0xFF) : 0u;
    const uint32_t rowX = liveA ? (uint32_t)((exit1 >> (8 * r)) & 0xFF) : 0u;
    bool bad = (rowE & (rowE - 1)) != 0u || (rowX & (rowX - 1)) != 0u;
    const uint64_t cX = liveB ? ((exit1 >> r) & col0) : 0ull, cE = liveB ? ((entry1 >> r) & col0) : 0ull;
    bad |= (cX & (cX - 1)) != 0ull || (cE & (cE - 1)) != 0ull;
    const uint32_t nxt1 = (in1 >> 1) | ((in1 & 1u) << (n1 - 1));
    const uint32_t nxt2 = (in2 >> 1) | ((in2 & 1u) << (n2 - 1));
    const uint32_t xrow = liveA ? (uint32_t)((X >> (8 * r)) & 0xFF) : 0u;
    float lane2 = ((nxt1 >> r) & 1u && liveA) ? c1r : 0.f;
    lane2 += ((nxt2 >> r) & 1u && liveB) ? c2r : 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) lane2 += ((xrow >> j) & 1u) ? term[j] : 0.f;
    const float twoA = gsum(gm, lane2);
    const float ai = 0.5f * twoA;
    const float U = a1 + a2 - ai;
    if (U < kThinRel * Lr * Lr) return false; // thin pair: float-float areas on the warp path

    // chunk of the vertex order from P1 edge r
    uint64_t c_lo = 0, c_hi = 0;
    uint32_t len = 0, qm = 0;
    if (liveA) {
        if ((in1 >> r) & 1u) {
            c_lo |= (uint64_t)r;
            ++len;
        }
        if (rowE) {
            c_lo |= (uint64_t)(0x80u | ((uint32_t)r << 3) | (uint32_t)(__ffs(rowE) - 1)) << (8 * len);
            ++len;
        }
        if (rowX) {
            const uint32_t jx = (uint32_t)(__ffs(rowX) - 1);
            c_lo |= (uint64_t)(0x80u | ((uint32_t)r << 3) | jx) << (8 * len);
            ++len;
            uint32_t j = (jx + 1 < (uint32_t)n2) ? jx + 1 : 0u;
            for (int m = 0; m < 8 && ((in2 >> j) & 1u) && !((qm >> j) & 1u); ++m) {
                qm |= 1u << j;
                const uint64_t code = 0x40u | j;
                if (len < 8) c_lo |= code << (8 * len);
                else c_hi |= code << (8 * (len - 8));
                ++len;
                j = (j + 1 < (uint32_t)n2) ? j + 1 : 0u;
            }
        }
    }
    uint32_t off = len;
#pragma unroll
    for (int d = 1; d < G; d <<= 1) {
        const uint32_t v = __shfl_up_sync(gm, off, d, G);
        if (r >= d) off += v;
    }
    const uint32_t total = __shfl_sync(gm, off, base + 7);
    off -= len;
    // one group OR for the P2 chain marks (8 bits) and the lane's own checks
    const uint32_t qb = gor32(gm, qm | (bad ? 0x100u : 0u));
    const uint32_t qall = qb & 0xFFu;
    bool bad_g = (qb >> 8) != 0u; // group-uniform from here on
    uint64_t s_lo = 0, s_hi = 0;
    if (len) {
        if (off == 0) {
            s_lo = c_lo;
            s_hi = c_hi;
        } else if (off < 8) {
            s_lo = c_lo << (8 * off);
            s_hi = (c_hi << (8 * off)) | (c_lo >> (64 - 8 * off));
        } else {
            s_hi = c_lo << (8 * (off - 8));
        }
    }
    s_lo = gor64(gm, s_lo);
    s_hi = gor64(gm, s_hi);
    const bool q_inside = X == 0 && in1 == 0;
    if (q_inside) {
        // P2 inside P1: the intersection is P2
        bad_g |= in2 != ((1u << n2) - 1u);
        s_lo = 0;
#pragma unroll
        for (int j = 0; j < 8; ++j) s_lo |= (j < n2) ? ((uint64_t)(0x40u | j) << (8 * j)) : 0ull;
        s_hi = 0;
    } else {
        bad_g |= total != cnt || qall != in2;
    }
    if (bad_g) return false;
    uint32_t start;
    if (in1) start = (uint32_t)(__ffs(in1) - 1);
    else if (in2) start = 0x40u | (uint32_t)(__ffs(in2) - 1);
    else {
        const int b = __ffsll((long long)X) - 1;
        start = 0x80u | ((uint32_t)(b / 8) << 3) | (uint32_t)(b % 8);
    }
    // slot of the smallest code (lowest byte equal to it), then rotate
    const uint64_t ones = 0x0101010101010101ull, highs = 0x8080808080808080ull, pat = ones * start;
    const uint64_t z0 = s_lo ^ pat, z1 = s_hi ^ pat;
    const uint64_t h0 = (z0 - ones) & ~z0 & highs, h1 = (z1 - ones) & ~z1 & highs;
    const uint32_t p0 = h0 ? (uint32_t)((__ffsll((long long)h0) - 1) >> 3)
                           : 8u + (uint32_t)((__ffsll((long long)h1) - 1) >> 3);
    // rotate the cnt-byte cycle left by p0 bytes
    typedef unsigned __int128 u128;
    u128 seq = ((u128)s_hi << 64) | (u128)s_lo;
    if (p0 && p0 < cnt) {
        const u128 keep = (cnt >= 16u) ? ~(u128)0 : (((u128)1 << (8u * cnt)) - 1u);
        seq = ((seq >> (8u * p0)) | (seq << (8u * (cnt - p0)))) & keep;
    }
    const uint64_t lo = (uint64_t)seq, hi = (uint64_t)(seq >> 64);
    out.w0 = lo | ((cnt < 8) ? (~0ull << (8 * cnt)) : 0ull);
    out.w1 = hi | ((cnt <= 8) ? ~0ull : ((cnt < 16) ? (~0ull << (8 * (cnt - 8))) : 0ull));
    out.nx = cnt;
    out.iou = (U > 0.f) ? ai / U : 0.f;
    out.ai = ai;
    out.a1 = a1;
    out.a2 = a2;
    return true;
}

// Group backward (shape derivative).  Returns 0, kDevBadFlags, or kSlow
// (group-uniform) when the pair must take the shoelace adjoint.  On success
// lane r holds the gradients of P1 vertex r and P2 vertex r (0 beyond counts).
template <typename LaneT, typename Adj>
__device__ __forceinline__ uint32_t bwd_group(const LaneT& L, Adj& adj, uint32_t nx, uint64_t w0, uint64_t w1,
                                              bool refine, float& g1x, float& g1y, float& g2x, float& g2y) {
    const unsigned gm = gmask();
    const int base = gbase();
    const int r = L.r, n1 = L.n1, n2 = L.n2;
    const bool liveA = r < n1, liveB = r < n2;
    g1x = g1y = g2x = g2y = 0.f;
    if (nx > 16u) return kDevBadFlags;
    // fewer than three vertices: an empty intersection, no piece on any edge
    const bool empty = nx < 3u;
    // decode slots r and r + 8 on lane r, then OR across the group
    uint32_t in1 = 0, in2 = 0, other = 0;
    uint64_t X = 0;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const uint32_t k = (uint32_t)r + 8u * h;
        const uint32_t c = (uint32_t)(((h ? w1 : w0) >> (8 * r)) & 0xFFull);
        const bool live = !empty && k < nx;
        const uint32_t kind = c >> 6, lo = c & 7u, ci = (c >> 3) & 7u, v = c & 0x3Fu;
        in1 |= (live && kind == 0u && v < 8u) ? (1u << v) : 0u;
        in2 |= (live && kind == 1u && v < 8u) ? (1u << v) : 0u;
        X |= (live && kind == 2u) ? (1ull << (ci * 8 + lo)) : 0ull;
        other |= (live && (kind == 3u || (kind < 2u && v >= 8u) ||
                           (kind == 2u && (ci >= (uint32_t)n1 || lo >= (uint32_t)n2)))) ? 1u : 0u;
    }
    // one group OR for the three small masks (8 + 8 + 1 bits)
    const uint32_t pk = gor32(gm, in1 | (in2 << 8) | (other << 16));
    in1 = pk & 0xFFu;
    in2 = (pk >> 8) & 0xFFu;
    other = pk >> 16;
    X = gor64(gm, X);
    if (other || (in1 >> n1) || (in2 >> n2)) return kDevBadFlags;
    const uint64_t col0 = col0_mask();
    const uint32_t rn1 = (r + 1 < n1) ? (uint32_t)(r + 1) : 0u, rn2 = (r + 1 < n2) ? (uint32_t)(r + 1) : 0u;
    const uint32_t rowX = liveA ? (uint32_t)((X >> (8 * r)) & 0xFF) : 0u;
    const uint64_t colX = liveB ? ((X >> r) & col0) : 0ull;
    bool ok = empty || (uint32_t)(__popc(in1) + __popc(in2) + __popcll(X)) == nx;
    {
        const uint32_t ra = (uint32_t)__popc(rowX), a0 = (in1 >> r) & 1u, a1 = (in1 >> rn1) & 1u;
        ok &= !liveA || ((a0 ^ a1) ? ra == 1u : (a0 ? ra == 0u : (ra == 0u || ra == 2u)));
        const uint32_t rb = (uint32_t)__popcll(colX), b0 = (in2 >> r) & 1u, b1 = (in2 >> rn2) & 1u;
        ok &= !liveB || ((b0 ^ b1) ? rb == 1u : (b0 ? rb == 0u : (rb == 0u || rb == 2u)));
    }
    if (gor32(gm, ok ? 0u : 1u)) return kSlow;

    const float kInf = __int_as_float(0x7f800000);
    // P1 edge r: parameters of its (at most two) crossings, with the P2
    // edges' data fetched from their lanes
    float t0 = kInf, t1 = -kInf;
    uint32_t rx = rowX;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int j = rx ? __ffs(rx) - 1 : 0;
        const bool has = rx != 0u;
        rx &= rx ? rx - 1u : 0u;
        const float bx = __shfl_sync(gm, L.bxr, base + j), by = __shfl_sync(gm, L.byr, base + j);
        const float ebx = __shfl_sync(gm, L.ebxr, base + j), eby = __shfl_sync(gm, L.ebyr, base + j);
        if (has) {
            const float dx = L.ax - bx, dy = L.ay - by;
            const float S = ebx * dy - eby * dx, D = L.eax * eby - L.eay * ebx;
            const float t = S * __fdividef(1.0f, D);
            t0 = fminf(t0, t);
            t1 = fmaxf(t1, t);
        }
    }
    t0 = ((in1 >> r) & 1u) ? 0.f : t0;
    t1 = ((in1 >> rn1) & 1u) ? 1.f : t1;
    // P2 edge r: parameters of its crossings, with the P1 edges' data fetched
    // from their lanes
    const float bxr = L.bxr, byr = L.byr, ebxr = L.ebxr, ebyr = L.ebyr;
    float u0 = kInf, u1 = -kInf;
    uint64_t cx = colX;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int i = cx ? (__ffsll((long long)cx) - 1) / 8 : 0;
        const bool has = cx != 0ull;
        cx &= cx ? cx - 1 : 0ull;
        const float ax = __shfl_sync(gm, L.ax, base + i), ay = __shfl_sync(gm, L.ay, base + i);
        const float eax = __shfl_sync(gm, L.eax, base + i), eay = __shfl_sync(gm, L.eay, base + i);
        if (has) {
            const float dx = ax - bxr, dy = ay - byr;
            const float T = eay * dx - eax * dy, D = eax * ebyr - eay * ebxr;
            const float u = -T * __fdividef(1.0f, D);
            u0 = fminf(u0, u);
            u1 = fmaxf(u1, u);
        }
    }
    u0 = ((in2 >> r) & 1u) ? 0.f : u0;
    u1 = ((in2 >> rn2) & 1u) ? 1.f : u1;
    const bool hasA = liveA && (((in1 >> r) & 1u) || rowX);
    const bool hasB = liveB && (((in2 >> r) & 1u) || colX);
    const float c1 = liveA ? L.ax * L.eay - L.ay * L.eax : 0.f;
    const float c2 = liveB ? bxr * ebyr - byr * ebxr : 0.f;
    const float twoA = gsum(gm, (hasA ? (t1 - t0) * c1 : 0.f) + (hasB ? (u1 - u0) * c2 : 0.f));
    const float a1 = 0.5f * gsum(gm, c1), a2 = 0.5f * gsum(gm, c2);
    const float ai = 0.5f * twoA;
    const float Lr = gmax(gm, fmaxf(liveA ? fmaxf(fabsf(L.ax), fabsf(L.ay)) : 0.f,
                                    liveB ? fmaxf(fabsf(bxr), fabsf(byr)) : 0.f));
    if (refine && !empty && ai < kTinyArea * Lr * Lr) return kSlow;
    float gai, ga1, ga2;
    if (!adj(ai, a1, a2, gai, ga1, ga2)) return 0u;
    const float h1 = 0.5f * ga1, h2 = 0.5f * ga2;
    const float I0a = hasA ? 0.5f * ((1.f - t0) * (1.f - t0) - (1.f - t1) * (1.f - t1)) : 0.f;
    const float I1a = hasA ? 0.5f * (t1 * t1 - t0 * t0) : 0.f;
    const float I0b = hasB ? 0.5f * ((1.f - u0) * (1.f - u0) - (1.f - u1) * (1.f - u1)) : 0.f;
    const float I1b = hasB ? 0.5f * (u1 * u1 - u0 * u0) : 0.f;
    const float wsa = liveA ? gai * I0a + h1 : 0.f, wea = liveA ? gai * I1a + h1 : 0.f;
    const float wsb = liveB ? gai * I0b + h2 : 0.f, web = liveB ? gai * I1b + h2 : 0.f;
    const float ex1 = wea * L.eay, ey1 = -wea * L.eax, ex2 = web * ebyr, ey2 = -web * ebxr;
    // vertex r receives the end contribution of edge r - 1 (wrapping at the count)
    const int pa = base + ((r == 0) ? n1 - 1 : r - 1), pb = base + ((r == 0) ? n2 - 1 : r - 1);
    const float px1 = __shfl_sync(gm, ex1, pa), py1 = __shfl_sync(gm, ey1, pa);
    const float px2 = __shfl_sync(gm, ex2, pb), py2 = __shfl_sync(gm, ey2, pb);
    g1x = liveA ? wsa * L.eay + px1 : 0.f;
    g1y = liveA ? -wsa * L.eax + py1 : 0.f;
    g2x = liveB ? wsb * ebyr + px2 : 0.f;
    g2y = liveB ? -wsb * ebxr + py2 : 0.f;
    return 0u;
}

} // namespace g8
} // namespace dgal
