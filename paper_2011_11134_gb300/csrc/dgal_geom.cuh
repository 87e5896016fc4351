// Device geometry for convex-polygon IoU on sm_103a: one thread owns one pair.
//
// Forward (paper Sec. II-B `intersect`, `area`, `iou`):
//   * the pair is moved to a local frame whose origin is P1's vertex 0, so the
//     FP32 orientation tests do not cancel at large coordinates;
//   * all vertex-vs-edge orientations S(i,j) = orient(b_j, b_j+1, a_i) and
//     T(i,j) = orient(a_i, a_i+1, b_j) are reduced to sign bitmasks; inside
//     tests, proper edge crossings and entry/exit directions are bit logic;
//   * the intersection polygon's vertex order comes from walking its boundary
//     (P1 vertex -> end of its P1 edge piece, crossing -> continue on the
//     polygon being entered), not from sorting, and starts at the smallest
//     code, so nx / xflags come out in the canonical form directly;
//   * the area is the shoelace sum grouped by edge pieces, rewritten so that
//     each inside vertex and each proper crossing adds one term
//     (fwd_generic); no vertex ordering and no crossing point is needed for
//     it;
//   * for quadrilaterals without counts the walk is table-driven: one 64-bit
//     table entry per edge gives that edge's block of codes.
//   With refinement, orientations too small for their FP32 sign take the
//   FP64 definition's sign, and exact zeros the sign under an infinitesimal
//   translation of P2 (tie_neg).  Thin pairs, pairs whose sign pattern is not
//   that of two convex polygons in general position, and (without
//   refinement) near-degenerate pairs take the warp-cooperative robust path
//   (candidate gathering and an angular sort; with refinement, FP64
//   orientation tests and float-float crossing parameters and areas).
//
// Backward (paper Sec. II-B `iou_grad`): the recorded codes rebuild the
// intersection vertices (crossings as a + t ea), the shoelace adjoint gives
// each vertex's gradient, and crossing gradients flow through t = S / D onto
// the four endpoints of the two edges.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace dgal {

constexpr float kDegenRel = 1e-5f; // near-degenerate threshold (relative to L^2, or to t, u in (0, 1))

// Routing threshold of the FP32 fast paths, relative to L^2 (L = largest
// |local coordinate| of the pair).  An orientation evaluated in the local
// frame as (c - b) x (a - b) differs from the exact orientation of the input
// points by at most 48 u L^2 (u = 2^-24) to first order: 16 u L^2 from
// rounding the three points into the local frame and 32 u L^2 from the four
// differences, two products and one subtraction (each difference bounded by
// 2L).  That is 2.9e-6 L^2, so every orientation with |value| > 5e-6 L^2 has
// its exact sign, and the fast path decides only those pairs.  Pairs with an
// orientation between this and kDegenRel are still reported near-degenerate.
constexpr float kRouteRel = 5e-6f;

// Thin-pair routing of the FP32 fast paths.  Their areas carry an absolute
// error of order u L^2 (each shoelace term is a difference of products of
// coordinates up to L), so the IoU error grows as u L^2 / U for a small union
// U.  An intersecting pair with U below this fraction of L^2 (thin or tiny
// polygons far apart in the pair's frame) is handed to the warp-cooperative
// path, whose rounding estimate takes such areas in float-float.  None of the
// IoU-loss rectangle pairs and about 0.05% of the intersecting convex-hull
// pairs are below it.
constexpr float kThinRel = 0.02f;

// device status bits (mirror include/dgal.h)
constexpr uint32_t kDevBadCount = 0x1u;
constexpr uint32_t kDevOverflow = 0x2u;
constexpr uint32_t kDevBadFlags = 0x4u;
constexpr uint32_t kDevBadOffsets = 0x8u;
constexpr uint32_t kDevTimeout = 0x10u;
constexpr uint32_t kDevNotConvex = 0x20u;

// flag bits of the C ABI
constexpr uint32_t kFlagRefine = 0x1u;
constexpr uint32_t kFlagPlain = 0x2u;

template <int K> struct MaskOf { typedef uint64_t T; };
template <> struct MaskOf<4> { typedef uint32_t T; };

// 2K one-byte codes, slot k in byte k.
template <int K> struct Codes {
    uint64_t w[(2 * K + 7) / 8];
};

template <int K> __device__ __forceinline__ void codes_fill(Codes<K>& c, uint64_t v) {
#pragma unroll
    for (int q = 0; q < (2 * K + 7) / 8; ++q) c.w[q] = v;
}

template <int K> __device__ __forceinline__ uint32_t code_at(const Codes<K>& c, uint32_t k) {
    if constexpr (K <= 4) {
        return (uint32_t)(c.w[0] >> (8u * k)) & 0xFFu;
    } else {
        uint64_t w = (k < 8u) ? c.w[0] : c.w[1];
        return (uint32_t)(w >> (8u * (k & 7u))) & 0xFFu;
    }
}

// Clears slot k to `code` (slot must hold 0xFF before).
template <int K> __device__ __forceinline__ void code_put(Codes<K>& c, uint32_t k, uint32_t code) {
    uint64_t m = ~((uint64_t)(0xFFu ^ code) << (8u * (k & 7u)));
    if constexpr (K <= 4) {
        c.w[0] &= m;
    } else {
        if (k < 8u) c.w[0] &= m; else c.w[1] &= m;
    }
}

template <typename T> __device__ __forceinline__ int ctz_(T m) {
    if constexpr (sizeof(T) == 8) return __ffsll((long long)m) - 1;
    else return __ffs((int)m) - 1;
}
template <typename T> __device__ __forceinline__ int popc_(T m) {
    if constexpr (sizeof(T) == 8) return __popcll(m);
    else return __popc(m);
}

// Three-operand minimum / maximum (one instruction on sm_100 and later).
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}
__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Shifts acc left by one and moves the sign bit of v into bit 0 (one funnel
// shift), so that sign masks are built without a shift and an OR per bit.
__device__ __forceinline__ uint32_t push_sign(uint32_t acc, float v) {
    return __funnelshift_l(__float_as_uint(v), acc, 1);
}

// Packed FP32 pairs (sm_100 and later): one instruction rounds two
// independent FP32 results, each exactly as the scalar add / sub / mul / fma
// would.  The pair loops below use them to form two columns (j, j + 1) of a
// row at a time, halving the issue slots of the orientation arithmetic.
__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 pa, pb, pd;\n\t"
        "mov.b64 pa, {%2, %3};\n\t"
        "mov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pd, pa, pb;\n\t"
        "mov.b64 {%0, %1}, pd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// P2 operands of edges j, j + 1 (lane x: edge j, lane y: edge j + 1).
struct ColPair {
    float2 bx, by, ebx, eby;
};
template <int K> __device__ __forceinline__ ColPair col_pair(const float (&bx)[K], const float (&by)[K],
                                                             const float (&ebx)[K], const float (&eby)[K], int h) {
    const int j = 2 * h;
    ColPair c;
    c.bx = f2(bx[j], bx[j + 1]);
    c.by = f2(by[j], by[j + 1]);
    c.ebx = f2(ebx[j], ebx[j + 1]);
    c.eby = f2(eby[j], eby[j + 1]);
    return c;
}

// One vertex-edge block for the two P2 edges of q against P1 vertex / edge i:
//   S  = orient(b_j, b_j+1, a_i)  = ebx_j dy + eby_j mx,
//   nT = -orient(a_i, a_i+1, b_j) = eax_i dy + eay_i mx,
//   D  = cross(ea_i, eb_j)        = eax_i eby_j - eay_i ebx_j,
//   nc = -cross(a_i, b_j)         = ay_i bx_j - ax_i by_j,
// with mx = bx_j - ax_i and dy = ay_i - by_j (the local differences of the
// scalar form, one of them negated, so that no P2 operand needs a negated
// copy).  Each lane's value is the scalar formula's: one rounded difference
// per coordinate, one rounded product and one fused multiply-add per
// orientation.  ORIGIN: a_i is the local origin (i = 0), so mx = bx and
// nc = 0 without arithmetic.  NC: form nc (the forward's area term).
struct Blk2 {
    float2 S, nT, D, nc;
};
template <bool ORIGIN, bool NC>
__device__ __forceinline__ Blk2 blk2(float ax, float ay, float eax, float eay, const ColPair& q) {
    Blk2 b;
    const float2 mx = ORIGIN ? q.bx : sub2(q.bx, f2(ax, ax));
    const float2 dy = sub2(f2(ay, ay), q.by);
    b.S = fma2(q.ebx, dy, mul2(q.eby, mx));
    b.nT = fma2(f2(eax, eax), dy, mul2(f2(eay, eay), mx));
    b.D = fma2(f2(eax, eax), q.eby, mul2(f2(-eay, -eay), q.ebx));
    if constexpr (NC) b.nc = ORIGIN ? f2(0.f, 0.f) : fma2(f2(ay, ay), q.bx, mul2(f2(-ax, -ax), q.by));
    return b;
}

// Value at dynamic index idx of a register array (select chain, no local memory).
template <int K> __device__ __forceinline__ float sel(const float (&a)[K], uint32_t idx) {
    float r = a[0];
#pragma unroll
    for (int m = 1; m < K; ++m) r = (idx == (uint32_t)m) ? a[m] : r;
    return r;
}

// Polygon loads: K x (x, y) as K/2 128-bit loads (16-byte aligned rows).
template <int K> __device__ __forceinline__ void load_poly(const float* __restrict__ p, float (&x)[K], float (&y)[K]) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int v = 0; v < K / 2; ++v) {
        float4 f = __ldg(q + v);
        x[2 * v] = f.x;
        y[2 * v] = f.y;
        x[2 * v + 1] = f.z;
        y[2 * v + 1] = f.w;
    }
}

// A pair in P1's local frame; edges wrap at the vertex counts.
template <int K> struct Geo {
    float ax[K], ay[K], bx[K], by[K];
    float eax[K], eay[K], ebx[K], eby[K];
    int n1, n2;
};

template <int K, bool COUNTS>
__device__ __forceinline__ void make_geo(const float (&px)[K], const float (&py)[K], const float (&qx)[K],
                                         const float (&qy)[K], int n1, int n2, Geo<K>& g) {
    const float ox = px[0], oy = py[0];
#pragma unroll
    for (int v = 0; v < K; ++v) {
        // P1's vertex 0 is the origin: exactly 0 for finite inputs, and
        // written as 0 so that the terms it would multiply drop out
        g.ax[v] = v ? px[v] - ox : 0.f;
        g.ay[v] = v ? py[v] - oy : 0.f;
        g.bx[v] = qx[v] - ox;
        g.by[v] = qy[v] - oy;
    }
#pragma unroll
    for (int v = 0; v < K; ++v) {
        float nax = g.ax[0], nay = g.ay[0], nbx = g.bx[0], nby = g.by[0];
        if (v + 1 < K) {
            bool w1 = COUNTS && (v + 1 >= n1);
            bool w2 = COUNTS && (v + 1 >= n2);
            nax = w1 ? g.ax[0] : g.ax[v + 1];
            nay = w1 ? g.ay[0] : g.ay[v + 1];
            nbx = w2 ? g.bx[0] : g.bx[v + 1];
            nby = w2 ? g.by[0] : g.by[v + 1];
        }
        g.eax[v] = nax - g.ax[v];
        g.eay[v] = nay - g.ay[v];
        g.ebx[v] = nbx - g.bx[v];
        g.eby[v] = nby - g.by[v];
    }
    g.n1 = COUNTS ? n1 : K;
    g.n2 = COUNTS ? n2 : K;
}

template <int K> struct FwdOut {
    Codes<K> codes;
    float iou;
    float ai, a1, a2;
    float L2; // squared coordinate scale of the pair (fast path)
    uint32_t nx;
    uint32_t degen; // bit 0 near-degenerate, bit 1 FP64 orientation tests used
    uint32_t err;   // device status bits
};

template <int K, bool COUNTS> __device__ __forceinline__ void input_areas(const Geo<K>& g, float& a1, float& a2) {
    float s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int v = 0; v < K; ++v) {
        float c1 = g.ax[v] * g.eay[v] - g.ay[v] * g.eax[v];
        float c2 = g.bx[v] * g.eby[v] - g.by[v] * g.ebx[v];
        s1 += (!COUNTS || v < g.n1) ? c1 : 0.f;
        s2 += (!COUNTS || v < g.n2) ? c2 : 0.f;
    }
    a1 = 0.5f * s1;
    a2 = 0.5f * s2;
}

template <int K, bool COUNTS> __device__ __forceinline__ float pair_scale(const Geo<K>& g) {
    float L = 0.f;
    if constexpr (!COUNTS) {
#pragma unroll
        for (int v = 0; v < K; ++v) {
            L = fmax3(L, fabsf(g.ax[v]), fabsf(g.ay[v]));
            L = fmax3(L, fabsf(g.bx[v]), fabsf(g.by[v]));
        }
    } else {
#pragma unroll
        for (int v = 0; v < K; ++v) {
            float la = fmaxf(fabsf(g.ax[v]), fabsf(g.ay[v]));
            float lb = fmaxf(fabsf(g.bx[v]), fabsf(g.by[v]));
            L = fmaxf(L, v < g.n1 ? la : 0.f);
            L = fmaxf(L, v < g.n2 ? lb : 0.f);
        }
    }
    return L;
}

// ------------------------------------------------------------ generic path

// orient(a, b, p) = cross(b - a, p - a) of three input points read from the
// unrounded FP32 inputs, in IEEE double without contraction and in the same
// operand order as the FP64 definition, so the value (and its sign) is the
// FP64 definition's.
__device__ __forceinline__ double orient_raw(const float* __restrict__ pa, int ia, int ib,
                                             const float* __restrict__ pp, int ip) {
    const float2 A = __ldg(reinterpret_cast<const float2*>(pa) + ia);
    const float2 B = __ldg(reinterpret_cast<const float2*>(pa) + ib);
    const float2 P = __ldg(reinterpret_cast<const float2*>(pp) + ip);
    const double bx = __dsub_rn((double)B.x, (double)A.x), by = __dsub_rn((double)B.y, (double)A.y);
    const double px = __dsub_rn((double)P.x, (double)A.x), py = __dsub_rn((double)P.y, (double)A.y);
    return __dsub_rn(__dmul_rn(bx, py), __dmul_rn(by, px));
}

// Sign of an orientation whose exact value is zero (a vertex on the line of
// an edge), taken as under an infinitesimal translation of P2 by
// (eps, eps^2).  With eb = b_j+1 - b_j and ea = a_i+1 - a_i,
//   S(i,j) = orient(b_j, b_j+1, a_i) becomes S + eby eps - ebx eps^2,
//   T(i,j) = orient(a_i, a_i+1, b_j) becomes T - eay eps + eax eps^2,
// so a zero S takes the sign of eby (of -ebx when eby = 0) and a zero T the
// sign of -eay (of eax when eay = 0).  The translated pair has no vertex on
// the line of any edge (that would need the edge parallel to (eps, eps^2)),
// so its signs are those of two convex polygons in general position, and
// since the intersection area is continuous, its clip evaluated at eps = 0
// gives the exact area.  The edge components come from the raw inputs: an
// FP32 difference of two floats is zero exactly when they are equal, so its
// sign is exact.  p1edge: the edge is P1's (a T orientation).  Returns 1 for
// a negative sign, 0 for a positive one, 2 for an edge of zero length (no
// decision).
__device__ __forceinline__ uint32_t tie_neg(const float* __restrict__ raw, int ia, int ib, bool p1edge) {
    const float2 A = __ldg(reinterpret_cast<const float2*>(raw) + ia);
    const float2 B = __ldg(reinterpret_cast<const float2*>(raw) + ib);
    const float ex = B.x - A.x, ey = B.y - A.y;
    if (ey != 0.f) return ((ey > 0.f) == p1edge) ? 1u : 0u;
    if (ex != 0.f) return ((ex < 0.f) == p1edge) ? 1u : 0u;
    return 2u;
}

// Sign repair for a pair of quadrilaterals (K = 4): `small` marks the
// orientations whose FP32 value is too small to trust (bit i*4+j: S(i,j) =
// orient(b_j, b_j+1, a_i); bit 16+i*4+j: T(i,j) = orient(a_i, a_i+1, b_j)),
// `neg` holds the FP32 signs in the same layout.  Each marked orientation is
// re-evaluated by orient_raw and its sign bit replaced; an exact zero takes
// the sign of the translated pair (tie_neg).  Returns the repaired signs, or
// bit 32 set when a zero sits on an edge of zero length.  Not inlined: it runs for well
// under 0.1% of random pairs, and keeping it out of line keeps the fast
// path's registers unchanged.
static __device__ __noinline__ uint64_t exact_signs4(const float* __restrict__ raw1, const float* __restrict__ raw2, int n1,
                                              int n2, uint32_t small, uint32_t neg) {
    while (small) {
        const int b = __ffs(small) - 1;
        small &= small - 1u;
        const int q = b & 15, i = q >> 2, j = q & 3;
        const int i1 = (i + 1 < n1) ? i + 1 : 0, j1 = (j + 1 < n2) ? j + 1 : 0;
        const double v = (b >= 16) ? orient_raw(raw1, i, i1, raw2, j) : orient_raw(raw2, j, j1, raw1, i);
        uint32_t ng = (v < 0.0) ? 1u : 0u;
        if (v == 0.0) {
            ng = (b >= 16) ? tie_neg(raw1, i, i1, true) : tie_neg(raw2, j, j1, false);
            if (ng > 1u) return 1ull << 32;
        }
        neg = ng ? (neg | (1u << b)) : (neg & ~(1u << b));
    }
    return neg;
}

// The sign repair of fwd_finish (K = 4): the pair's local frame is rebuilt
// from the raw inputs (so the caller need not keep its geometry live), every
// orientation within 3x the routing threshold thr is marked (the marks are
// taken on this recomputation, which may round differently from the caller's
// values by up to twice the FP32 error bound, so the margin covers every
// value that was under the threshold), and exact_signs4 takes the FP64
// definition's sign for each.  neg: the caller's sign bits (S at bit 4i + j,
// T at bit 16 + 4i + j).  Not inlined: it runs for well under 0.1% of pairs.
static __device__ __noinline__ uint64_t refine_signs4(const float* __restrict__ raw1, const float* __restrict__ raw2,
                                                      int n1, int n2, float thr, uint32_t neg) {
    float px[4], py[4], qx[4], qy[4];
    const float4* a = reinterpret_cast<const float4*>(raw1);
    const float4* b = reinterpret_cast<const float4*>(raw2);
#pragma unroll
    for (int v = 0; v < 2; ++v) {
        const float4 f = __ldg(a + v), h = __ldg(b + v);
        px[2 * v] = f.x; py[2 * v] = f.y; px[2 * v + 1] = f.z; py[2 * v + 1] = f.w;
        qx[2 * v] = h.x; qy[2 * v] = h.y; qx[2 * v + 1] = h.z; qy[2 * v + 1] = h.w;
    }
    const float ox = px[0], oy = py[0];
    float ax[4], ay[4], bx[4], by[4], eax[4], eay[4], ebx[4], eby[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        ax[v] = v ? px[v] - ox : 0.f;
        ay[v] = v ? py[v] - oy : 0.f;
        bx[v] = qx[v] - ox;
        by[v] = qy[v] - oy;
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int w1 = (v + 1 < n1) ? v + 1 : 0, w2 = (v + 1 < n2) ? v + 1 : 0;
        eax[v] = (w1 ? px[w1] - ox : 0.f) - ax[v];
        eay[v] = (w1 ? py[w1] - oy : 0.f) - ay[v];
        ebx[v] = (qx[w2] - ox) - bx[v];
        eby[v] = (qy[w2] - oy) - by[v];
    }
    const float wide = 3.f * thr;
    uint32_t small = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const bool valid = i < n1 && j < n2;
            const float dx = ax[i] - bx[j], dy = ay[i] - by[j];
            const float sv = ebx[j] * dy - eby[j] * dx;
            const float t = eay[i] * dx - eax[i] * dy;
            small |= (valid && !(fabsf(sv) > wide)) ? (1u << (i * 4 + j)) : 0u;
            small |= (valid && !(fabsf(t) > wide)) ? (1u << (16 + i * 4 + j)) : 0u;
        }
    }
    return exact_signs4(raw1, raw2, n1, n2, small, neg);
}

// 2K code bytes as one integer (byte k = slot k).
template <int K> struct SeqOf { typedef uint64_t T; };
template <> struct SeqOf<8> { typedef unsigned __int128 T; };

// Bytes 0x40 | ((s + m) mod n) for m < len, packed from byte 0: the codes of a
// chain of consecutive P2 vertices starting at s.
template <int K, bool COUNTS> __device__ __forceinline__ uint64_t q_chain_bytes(uint32_t s, uint32_t len, uint32_t n) {
    if constexpr (K == 4 && !COUNTS) {
        const uint32_t w = __funnelshift_r(0x43424140u, 0x43424140u, 8u * s);
        return len >= 4u ? (uint64_t)w : (uint64_t)(w & ((1u << (8u * len)) - 1u));
    } else {
        uint64_t c = 0;
#pragma unroll
        for (int m = 0; m < K; ++m) {
            uint32_t v = s + (uint32_t)m;
            v -= (v >= n) ? n : 0u;
            c |= ((uint32_t)m < len) ? ((uint64_t)(0x40u | v) << (8 * m)) : 0ull;
        }
        return c;
    }
}

// Table-driven walk for a pair of quadrilaterals without counts.  The block
// of codes that P1 edge i contributes to the boundary walk (its start vertex
// if inside P2, its entry crossing, its exit crossing, then the chain of P2
// vertices inside P1 that follows the exit) depends only on
//   idx = vI | rowE << 1 | rowX << 5 | in2 << 9
// (vI: start vertex inside; rowE / rowX: the edge's entry / exit crossings,
// bit j = P2 edge j; in2: P2 vertices inside P1).  Entry idx holds:
//   bits 0..39  the block's code bytes with the edge number left out (vertex
//               byte 0, crossing bytes 0x80 | j, chain bytes 0x40 | j);
//   bits 40..42 the block's length; bit 43: byte 0 is the start vertex;
//   bit 44      the pattern is impossible for two convex polygons in general
//               position (two entries or exits on one edge, an entry after an
//               inside start, a chain of every P2 vertex);
//   bits 48..51 the P2 vertices of the chain (to check that no P2 vertex is
//               emitted twice).
// The kernel adds the edge number (i to the vertex byte, i << 3 to crossing
// bytes) and appends the block at the running position.  Generated at
// compile time; 64 KB, read through L1.
struct WalkLut4 {
    unsigned long long e[8192];
};
constexpr int lut_ctz4(uint32_t m) { return (m & 1u) ? 0 : (m & 2u) ? 1 : (m & 4u) ? 2 : 3; }
constexpr int lut_popc4(uint32_t m) {
    return (int)(m & 1u) + (int)((m >> 1) & 1u) + (int)((m >> 2) & 1u) + (int)((m >> 3) & 1u);
}
constexpr unsigned long long walk_entry4(uint32_t idx) {
    const uint32_t vI = idx & 1u, rowE = (idx >> 1) & 15u, rowX = (idx >> 5) & 15u, in2 = (idx >> 9) & 15u;
    bool bad = lut_popc4(rowE) > 1 || lut_popc4(rowX) > 1 || (vI && rowE);
    unsigned long long bytes = 0;
    uint32_t sz = vI, cm = 0;
    if (rowE) {
        bytes |= (unsigned long long)(0x80u | (uint32_t)lut_ctz4(rowE)) << (8 * sz);
        ++sz;
    }
    if (rowX) {
        const uint32_t jx = (uint32_t)lut_ctz4(rowX);
        bytes |= (unsigned long long)(0x80u | jx) << (8 * sz);
        ++sz;
        uint32_t len = 0;
        while (len < 4u && ((in2 >> ((jx + 1u + len) & 3u)) & 1u)) {
            const uint32_t j = (jx + 1u + len) & 3u;
            bytes |= (unsigned long long)(0x40u | j) << (8 * sz);
            ++sz;
            cm |= 1u << j;
            ++len;
        }
        bad = bad || len >= 4u;
    }
    if (bad || sz > 5u) return 1ull << 44;
    return bytes | ((unsigned long long)sz << 40) | ((unsigned long long)vI << 43) | ((unsigned long long)cm << 48);
}
constexpr WalkLut4 make_walk_lut4() {
    WalkLut4 L{};
    for (uint32_t i = 0; i < 8192u; ++i) L.e[i] = walk_entry4(i);
    return L;
}
static __device__ const WalkLut4 g_walk_lut4 = make_walk_lut4();

template <int K, bool COUNTS>
__device__ __forceinline__ bool fwd_finish(const Geo<K>& g, float L, typename MaskOf<K>::T neg_s,
                                           typename MaskOf<K>::T neg_t, float minabs, const float (&Av)[K <= 4 ? K * K : 1],
                                           const float (&cv)[2][K], FwdOut<K>& o, const float* __restrict__ raw1,
                                           const float* __restrict__ raw2);

// Returns false when the pair must take the robust path: some orientation is
// within the near-degenerate threshold (|orient| <= 1e-5 L^2), or the sign
// pattern is not that of two convex polygons in general position.  While every
// |orient| exceeds that threshold (which is far above the FP32 rounding of the
// local-frame values), every sign is exact, so the inside tests, crossings and
// the vertex order are exactly those of the FP64 definition.  On success fills
// o.codes, o.nx and o.ai.
//
// raw1, raw2 (optional, K = 4): the pair's unrounded input polygons.  When
// given, a pair with orientations under the routing threshold is not handed
// back: those orientations take the FP64 definition's sign (exact_signs4), an
// exact zero (a vertex on the line of an edge) the sign under an
// infinitesimal translation of P2 (tie_neg), and only a zero-length edge
// hands the pair back.  Their FP32 values still place the crossing points: an
// FP32 orientation is
// within 2.9e-6 L^2 of the exact one, which moves a crossing point along its
// P1 edge and changes the intersection area by at most about 1.5e-6 L^2 per
// crossing, whatever the crossing angle (the same bound as for any pair of
// the fast path).  The pair is still reported near-degenerate.
template <int K, bool COUNTS>
__device__ __forceinline__ bool fwd_generic(const Geo<K>& g, FwdOut<K>& o, const float* __restrict__ raw1 = nullptr,
                                            const float* __restrict__ raw2 = nullptr) {
    typedef typename MaskOf<K>::T M;
    constexpr int KK = K * K;
    const int n1 = g.n1, n2 = g.n2;
    const float L = pair_scale<K, COUNTS>(g);

    // Orientation values: S(i,j) = orient(b_j, b_j+1, a_i), T(i,j) =
    // orient(a_i, a_i+1, b_j).  For K = 4 the loop also forms each pair of
    // edges' crossing term of the area (used below where (i, j) is a proper
    // crossing); for K = 8 the terms are formed later.
    constexpr bool KEEP = (K <= 4);
    float Av[KEEP ? KK : 1];
    M neg_s = 0, neg_t = 0;
    float minabs = __int_as_float(0x7f800000);
    if constexpr (K == 4) {
        // two P2 edges (j, j + 1) per packed instruction
        ColPair cp[K / 2];
#pragma unroll
        for (int h = 0; h < K / 2; ++h) cp[h] = col_pair<K>(g.bx, g.by, g.ebx, g.eby, h);
        // highest (i, j) first, so that push_sign leaves S(i,j)'s sign in
        // bit i * 4 + j
#pragma unroll
        for (int i = K - 1; i >= 0; --i) {
#pragma unroll
            for (int h = K / 2 - 1; h >= 0; --h) {
                const int j = 2 * h;
                Blk2 b;
                if (i == 0) b = blk2<true, true>(0.f, 0.f, g.eax[0], g.eay[0], cp[h]);
                else b = blk2<false, true>(g.ax[i], g.ay[i], g.eax[i], g.eay[i], cp[h]);
                // (c D + S T) / |D| = (-c D + S (-T)) / -|D|
                const float2 num = fma2(b.nc, b.D, mul2(b.S, b.nT));
                const float2 A =
                    mul2(num, f2(__fdividef(1.0f, -fabsf(b.D.x)), __fdividef(1.0f, -fabsf(b.D.y))));
                Av[i * K + j] = A.x;
                Av[i * K + j + 1] = A.y;
                const bool valid1 = !COUNTS || (i < n1 && j + 1 < n2);
                const bool valid0 = !COUNTS || (i < n1 && j < n2);
                minabs = valid1 ? fmin3(minabs, fabsf(b.S.y), fabsf(b.nT.y)) : minabs;
                minabs = valid0 ? fmin3(minabs, fabsf(b.S.x), fabsf(b.nT.x)) : minabs;
                neg_s = (M)push_sign(push_sign((uint32_t)neg_s, b.S.y), b.S.x);
                neg_t = (M)push_sign(push_sign((uint32_t)neg_t, b.nT.y), b.nT.x);
            }
        }
        // the bits of -T are set where T > 0; a zero T has |T| <= the routing
        // threshold, so its bit is never used as it stands
        neg_t = ~neg_t & (M)0xFFFFu;
    } else {
#pragma unroll
        for (int i = 0; i < K; ++i) {
#pragma unroll
            for (int j = 0; j < K; ++j) {
                const float dx = g.ax[i] - g.bx[j], dy = g.ay[i] - g.by[j];
                const float s = g.ebx[j] * dy - g.eby[j] * dx;
                const float t = g.eay[i] * dx - g.eax[i] * dy;
                const bool valid = !COUNTS || (i < n1 && j < n2);
                minabs = fminf(minabs, valid ? fminf(fabsf(s), fabsf(t)) : __int_as_float(0x7f800000));
                neg_s |= (M)(__float_as_uint(s) >> 31) << (i * K + j);
                neg_t |= (M)(__float_as_uint(t) >> 31) << (i * K + j);
            }
        }
    }
    float cv[2][K]; // cross(a_v, ea_v), cross(b_v, eb_v): the vertex terms of the area
#pragma unroll
    for (int v = 0; v < K; ++v) {
        cv[0][v] = g.ax[v] * g.eay[v] - g.ay[v] * g.eax[v];
        cv[1][v] = g.bx[v] * g.eby[v] - g.by[v] * g.ebx[v];
    }
    return fwd_finish<K, COUNTS>(g, L, neg_s, neg_t, minabs, Av, cv, o, raw1, raw2);
}

// The part of fwd_generic after the orientation values: the sign repair (with
// raw1, raw2), the masks, the inside tests, the area and the vertex order.
// L: the pair's scale; neg_s, neg_t: sign bits of S(i,j), T(i,j) at bit
// i K + j; minabs: the smallest |S|, |T| of the valid entries; Av: the
// crossing terms of the area (K = 4; unused for K = 8); cv: the vertex terms.
template <int K, bool COUNTS>
__device__ __forceinline__ bool fwd_finish(const Geo<K>& g, float L, typename MaskOf<K>::T neg_s,
                                           typename MaskOf<K>::T neg_t, float minabs, const float (&Av)[K <= 4 ? K * K : 1],
                                           const float (&cv)[2][K], FwdOut<K>& o, const float* __restrict__ raw1,
                                           const float* __restrict__ raw2) {
    typedef typename MaskOf<K>::T M;
    typedef typename SeqOf<K>::T Sq;
    constexpr int KK = K * K;
    constexpr int C = 2 * K;
    constexpr M kRow0 = (M)((1ull << K) - 1);
    constexpr bool KEEP = (K <= 4);
    M col0 = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) col0 |= (M)1 << (i * K);
    const int n1 = g.n1, n2 = g.n2;
    const float thr = kRouteRel * L * L;
    if (!(L > 0.f)) return false;
    uint32_t refined = 0u;
    if (!(minabs > thr)) {
        if constexpr (!KEEP) {
            return false;
        } else {
            if (raw1 == nullptr) return false;
            const uint64_t r = refine_signs4(raw1, raw2, n1, n2, thr, (uint32_t)neg_s | ((uint32_t)neg_t << 16));
            if (r >> 32) return false;
            neg_s = (M)(r & 0xFFFFu);
            neg_t = (M)((r >> 16) & 0xFFFFu);
            refined = 2u;
        }
    }
    o.degen = ((minabs <= kDegenRel * L * L) ? 1u : 0u) | refined;

    M V = (M)~(M)0;
    if constexpr (KK < 8 * (int)sizeof(M)) V = (M)((1ull << KK) - 1);
    M sp, tp, sp_next, tp_next;
    if constexpr (!COUNTS) {
        sp = ~neg_s & V;
        tp = ~neg_t & V;
        sp_next = (sp >> K) | ((sp & kRow0) << (K * (K - 1)));
        tp_next = ((tp >> 1) & ~(col0 << (K - 1))) | ((tp & col0) << (K - 1));
    } else {
        M rows = 0, cols = 0;
#pragma unroll
        for (int i = 0; i < K; ++i) rows |= (i < n1) ? (kRow0 << (i * K)) : (M)0;
#pragma unroll
        for (int j = 0; j < K; ++j) cols |= (j < n2) ? (col0 << j) : (M)0;
        V = rows & cols;
        sp = ~neg_s & V;
        tp = ~neg_t & V;
        sp_next = ((sp >> K) & ~(kRow0 << (K * (n1 - 1)))) | ((sp & kRow0) << (K * (n1 - 1)));
        tp_next = ((tp >> 1) & ~(col0 << (n2 - 1))) | ((tp & col0) << (n2 - 1));
    }
    const M X = (sp ^ sp_next) & (tp ^ tp_next) & V; // proper crossings (i, j)
    const M entry1 = X & ~sp;                         // P1 enters P2 there (a_i outside edge j)
    const M exit1 = X & sp;                           // P1 leaves P2 there
    if ((X & tp) != entry1) return false;             // P2 leaves P1 exactly where P1 enters P2

    // inside tests
    uint32_t in1 = 0, in2 = 0;
    if constexpr (K == 4 && !COUNTS) {
        // in1 bit i: row i of sp all set; in2 bit j: column j of tp all set
        uint32_t r = (uint32_t)sp & ((uint32_t)sp >> 1);
        r &= r >> 2;                                        // bit 4i: row i full
        in1 = (((r & 0x1111u) * 0x1248u) >> 12) & 15u;      // bits 0, 4, 8, 12 -> 0..3
        uint32_t c = (uint32_t)tp & ((uint32_t)tp >> 8);
        c &= c >> 4;                                        // bit j: column j full
        in2 = c & 15u;
    } else {
        const M colsFull = COUNTS ? (M)((1ull << n2) - 1) : kRow0;
        M rowsCol = 0;
#pragma unroll
        for (int i = 0; i < K; ++i) rowsCol |= (!COUNTS || i < n1) ? ((M)1 << (i * K)) : (M)0;
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const bool ok = ((sp >> (i * K)) & colsFull) == colsFull;
            in1 |= ((!COUNTS || i < n1) && ok) ? (1u << i) : 0u;
            const bool ok2 = ((tp >> i) & rowsCol) == rowsCol;
            in2 |= ((!COUNTS || i < n2) && ok2) ? (1u << i) : 0u;
        }
    }

    const uint32_t cnt = (uint32_t)(__popc(in1) + __popc(in2) + popc_(X));
    o.nx = 0;
    o.ai = 0.f;
    codes_fill<K>(o.codes, ~0ull);
    if (cnt == 0u) return true;
    if (cnt < 3u || cnt > (uint32_t)C) return false;

    const uint32_t n1m = COUNTS ? (uint32_t)n1 : (uint32_t)K;
    const uint32_t n2m = COUNTS ? (uint32_t)n2 : (uint32_t)K;
    // Area: the shoelace of the intersection grouped by edge pieces.  A piece
    // of P1 edge i runs between two points s, e of the line a_i + t ea_i, so
    // cross(s, e) = cross(a_i, e) - cross(a_i, s); likewise a piece of P2 edge
    // j with b_j.  Summing over pieces, every inside vertex a_i+1 adds
    // cross(a_i, ea_i) (the end of a piece at t = 1), every inside b_j+1 adds
    // cross(b_j, eb_j), and every crossing w of P1 edge i and P2 edge j adds
    // s cross(a_i - b_j, w), s = +1 where P1 leaves P2 (a P1 piece ends and a
    // P2 piece starts at w) and -1 where it enters.  With w = a_i + (S / D)
    // ea_i, S = S(i,j), T = T(i,j) = cross(a_i - b_j, ea_i), D = cross(ea_i,
    // eb_j), and s = sign(D) at a proper crossing, the crossing adds
    //   (cross(a_i, b_j) D + S T) / |D|.
    // The crossing point is one point for both of its pieces (no gap opens
    // between a P1 and a P2 parameter), and since |S| < |D| and |T| < |D| at a
    // proper crossing, the FP32 error of each term is of order u L^2 however
    // nearly parallel the two edges are.  No crossing point is formed.
    float twoA = 0.f;
    {
        uint32_t nxt1, nxt2; // bit v: vertex v + 1 (mod count) is inside
        if constexpr (!COUNTS) {
            nxt1 = (in1 >> 1) | ((in1 & 1u) << (K - 1));
            nxt2 = (in2 >> 1) | ((in2 & 1u) << (K - 1));
        } else {
            nxt1 = (in1 >> 1) | ((in1 & 1u) << (n1m - 1u));
            nxt2 = (in2 >> 1) | ((in2 & 1u) << (n2m - 1u));
        }
#pragma unroll
        for (int v = 0; v < K; ++v) {
            twoA += ((nxt1 >> v) & 1u) ? cv[0][v] : 0.f;
            twoA += ((nxt2 >> v) & 1u) ? cv[1][v] : 0.f;
        }
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int bit = i * K + j;
            if constexpr (KEEP) {
                twoA += ((X >> bit) & 1u) ? Av[bit] : 0.f;
            } else {
                const float dx = g.ax[i] - g.bx[j], dy = g.ay[i] - g.by[j];
                const float S = g.ebx[j] * dy - g.eby[j] * dx;
                const float T = g.eay[i] * dx - g.eax[i] * dy;
                const float D = g.eax[i] * g.eby[j] - g.eay[i] * g.ebx[j];
                const float c = g.ax[i] * g.by[j] - g.ay[i] * g.bx[j];
                const float r = ((X >> bit) & 1u) ? __fdividef(1.0f, fabsf(D)) : 0.f;
                twoA = fmaf(fmaf(c, D, S * T), r, twoA);
            }
        }
    }

    // Vertex order: walk P1's edges in order.  Edge i contributes its start
    // vertex (if inside P2), its entry crossing, its exit crossing and, after
    // an exit, the chain of P2 vertices inside P1 that the boundary follows
    // until P2 leaves P1 again.  The result is the counter-clockwise cycle;
    // it is rotated so that the smallest code comes first.
    uint32_t start;
    if (in1) start = (uint32_t)(__ffs(in1) - 1);
    else if (in2) start = 0x40u | (uint32_t)(__ffs(in2) - 1);
    else {
        const int b = ctz_(X);
        start = 0x80u | ((uint32_t)(b / K) << 3) | (uint32_t)(b % K);
    }
    Sq seq = 0;
    uint32_t pos = 0, p0 = 0, qmask = 0;
    bool bad = false;
    if constexpr (K == 4 && !COUNTS) {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const uint32_t idx = ((in1 >> i) & 1u) | (((uint32_t)(entry1 >> (i * K)) & 15u) << 1) |
                                 (((uint32_t)(exit1 >> (i * K)) & 15u) << 5) | (in2 << 9);
            const unsigned long long e = __ldg(&g_walk_lut4.e[idx]);
            const uint32_t lo = (uint32_t)e, hi = (uint32_t)(e >> 32);
            // edge number into the vertex byte (i) and the crossing bytes (i << 3)
            const uint32_t mult = ((lo >> 4) & 0x080808u) | ((hi >> 11) & 1u);
            const uint64_t blk = ((uint64_t)(hi & 0xFFu) << 32) | (uint64_t)(lo + (uint32_t)i * mult);
            const uint32_t cm = (hi >> 16) & 15u;
            bad |= (((hi >> 12) & 1u) | (qmask & cm)) != 0u;
            qmask |= cm;
            seq |= (Sq)blk << (8u * (pos & 7u));
            pos += (hi >> 8) & 7u;
        }
        if (X == 0 && in1 == 0) {
            // P2 inside P1: the intersection is P2
            bad |= in2 != 15u;
            seq = (Sq)0x43424140u;
            pos = 4u;
            qmask = in2;
        }
        // position of the smallest code: the zero byte of seq ^ start (codes
        // are distinct; bytes past the walk are 0, which only matches start
        // 0, P1 vertex 0, and that one is emitted first)
        const uint64_t x = (uint64_t)seq ^ (0x0101010101010101ull * (uint64_t)start);
        const uint64_t z = (x - 0x0101010101010101ull) & ~x & 0x8080808080808080ull;
        bad |= z == 0ull;
        p0 = ((uint32_t)__ffsll((long long)z) - 1u) >> 3;
    } else {
        const uint32_t jmin = (uint32_t)(__ffs(in2 | 0x100u) - 1);
        const uint32_t fullq = (1u << n2m) - 1u;
    #pragma unroll
        for (int i = 0; i < K; ++i) {
            if (COUNTS && i >= n1) break;
            if ((in1 >> i) & 1u) {
                p0 = ((uint32_t)i == start) ? pos : p0;
                seq |= (Sq)i << (8u * (pos & (C - 1)));
                ++pos;
            }
            const M rowE = (entry1 >> (i * K)) & kRow0;
            const M rowX = (exit1 >> (i * K)) & kRow0;
            bad |= ((rowE & (rowE - 1)) | (rowX & (rowX - 1))) != 0;
            if (rowE) {
                const uint32_t c = 0x80u | ((uint32_t)i << 3) | (uint32_t)ctz_(rowE);
                p0 = (c == start) ? pos : p0;
                seq |= (Sq)c << (8u * (pos & (C - 1)));
                ++pos;
            }
            if (rowX) {
                const uint32_t jx = (uint32_t)ctz_(rowX);
                const uint32_t c = 0x80u | ((uint32_t)i << 3) | jx;
                p0 = (c == start) ? pos : p0;
                seq |= (Sq)c << (8u * (pos & (C - 1)));
                ++pos;
                // P2 vertices jx+1, jx+2, ... (mod n2) while inside P1
                const uint32_t sh = (jx + 1u >= n2m) ? jx + 1u - n2m : jx + 1u;
                const uint32_t rot = sh ? (((in2 >> sh) | (in2 << (n2m - sh))) & fullq) : in2;
                const uint32_t len = (uint32_t)(__ffs(~rot) - 1);
                bad |= len >= n2m;
                const uint32_t lm = (1u << len) - 1u;
                const uint32_t cm = sh ? (((lm << sh) | (lm >> (n2m - sh))) & fullq) : lm;
                bad |= (qmask & cm) != 0u;
                qmask |= cm;
                if ((start >> 6) == 1u && ((cm >> jmin) & 1u)) p0 = pos + ((jmin + n2m - sh) % n2m);
                if (len) seq |= (Sq)q_chain_bytes<K, COUNTS>(sh, len, n2m) << (8u * (pos & (C - 1)));
                pos += len;
            }
        }
        if (X == 0 && in1 == 0) {
            // P2 inside P1: the intersection is P2
            bad |= in2 != fullq;
            seq = (Sq)q_chain_bytes<K, COUNTS>(0u, n2m, n2m);
            pos = n2m;
            qmask = in2;
            p0 = 0;
        }
    }
    if (bad || pos != cnt || qmask != in2) return false;
    if (p0) seq = (seq >> (8u * p0)) | (seq << (8u * (cnt - p0)));
    if (cnt < (uint32_t)C) seq = (seq & (((Sq)1 << (8u * cnt)) - 1)) | ~(((Sq)1 << (8u * cnt)) - 1);
    if constexpr (K == 4) {
        o.codes.w[0] = (uint64_t)seq;
    } else {
        o.codes.w[0] = (uint64_t)seq;
        o.codes.w[1] = (uint64_t)(seq >> 64);
    }
    o.nx = cnt;
    o.ai = 0.5f * twoA;
    o.L2 = L * L;
    return true;
}

// ------------------------------------------------------------- robust path

__device__ __forceinline__ double orient64(double ax, double ay, double bx, double by, double px, double py) {
    // no contraction: x*y - y*x is exactly zero, so exact collinearity of
    // shared float vertices is kept
    return __dsub_rn(__dmul_rn(__dsub_rn(bx, ax), __dsub_rn(py, ay)), __dmul_rn(__dsub_rn(by, ay), __dsub_rn(px, ax)));
}
__device__ __forceinline__ float orient32nc(float ax, float ay, float bx, float by, float px, float py) {
    return __fsub_rn(__fmul_rn(__fsub_rn(bx, ax), __fsub_rn(py, ay)), __fmul_rn(__fsub_rn(by, ay), __fsub_rn(px, ax)));
}

// Monotone stand-in for the polar angle of (dx, dy), in [0, 4).
__device__ __forceinline__ float pseudo_angle(float dx, float dy) {
    float s = fabsf(dx) + fabsf(dy);
    if (s == 0.f) return 0.f;
    float r = dy / s;
    if (dx >= 0.f) return dy >= 0.f ? r : 4.f + r;
    return 2.f - r;
}

// ------------------------------------------------------------ float-float
//
// A float-float number hi + lo carries about 48 significant bits with FP32
// instructions only: sums by the error-free two-sum, products with the FMA
// residual, a quotient refined by one correction step (the classic
// double-single arithmetic of Dekker and of Knuth's two-sum).  The warp
// paths take their accurate areas and shoelace adjoints in it, so that FP64
// stays with the orientation tests.

struct ff {
    float hi, lo;
    __device__ __forceinline__ ff() : hi(0.f), lo(0.f) {}
    __device__ __forceinline__ ff(float f) : hi(f), lo(0.f) {}
    __device__ __forceinline__ ff(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ explicit operator float() const { return hi + lo; }
};

// s + e = a + b exactly
__device__ __forceinline__ ff ff_two_sum(float a, float b) {
    const float s = a + b, bb = s - a;
    return ff(s, (a - (s - bb)) + (b - bb));
}
// the same for |a| >= |b| (or a = 0)
__device__ __forceinline__ ff ff_quick(float a, float b) {
    const float s = a + b;
    return ff(s, b - (s - a));
}
__device__ __forceinline__ ff operator+(ff x, ff y) {
    ff s = ff_two_sum(x.hi, y.hi);
    const ff t = ff_two_sum(x.lo, y.lo);
    s = ff_quick(s.hi, s.lo + t.hi);
    return ff_quick(s.hi, s.lo + t.lo);
}
__device__ __forceinline__ ff operator-(ff x) { return ff(-x.hi, -x.lo); }
__device__ __forceinline__ ff operator-(ff x, ff y) { return x + (-y); }
__device__ __forceinline__ ff operator*(ff x, ff y) {
    const float p = x.hi * y.hi;
    float e = fmaf(x.hi, y.hi, -p);
    e = fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e));
    return ff_quick(p, e);
}
__device__ __forceinline__ ff operator/(ff x, ff y) {
    const float q1 = x.hi / y.hi;
    const ff r = x - y * ff(q1);
    return ff_quick(q1, r.hi / y.hi);
}
__device__ __forceinline__ ff& operator+=(ff& x, ff y) { return x = x + y; }
__device__ __forceinline__ bool operator>(ff x, ff y) { return x.hi > y.hi || (x.hi == y.hi && x.lo > y.lo); }
__device__ __forceinline__ bool operator!=(ff x, ff y) { return x.hi != y.hi || x.lo != y.lo; }

// Warp shuffles of float and float-float values.
__device__ __forceinline__ float shfl(unsigned m, float v, int src) { return __shfl_sync(m, v, src); }
__device__ __forceinline__ ff shfl(unsigned m, ff v, int src) {
    return ff(__shfl_sync(m, v.hi, src), __shfl_sync(m, v.lo, src));
}
__device__ __forceinline__ float shfl_xor(unsigned m, float v, int off) { return __shfl_xor_sync(m, v, off); }
__device__ __forceinline__ ff shfl_xor(unsigned m, ff v, int off) {
    return ff(__shfl_xor_sync(m, v.hi, off), __shfl_xor_sync(m, v.lo, off));
}

// ------------------------------------------------- warp-cooperative robust path
//
// All 32 lanes of a warp work on one pair, with the candidate rules of the
// definition (inclusive vertex tests, strict crossings, exact duplicates
// dropped, angular order rotated to the smallest code).  Each orientation test
// runs on its own lane, in FP32 in the local frame and, when refining and the
// FP32 value is too small for its sign to be certain, in FP64 from the raw
// inputs (exact signs); the signs are combined by ballot, each candidate vertex is computed
// on its own lane (a crossing's parameters from the orientation values of the
// lanes that tested its edges), candidates are ranked by comparing against
// every other lane, and the areas are shuffle reductions of shoelace terms.
// The areas are taken in FP32 with an estimate of their rounding error; when
// refining and that estimate is not far below the IoU tolerance (slivers,
// tiny intersections), they are taken again in float-float about the
// candidates' centroid, with every crossing placed from float-float
// orientations.  GB300's FP64 rate is a small fraction of its FP32 rate, and
// FP64 is kept to the orientation tests.  The result is returned in every
// lane.

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return __shfl_sync(0xffffffffu, v, 0); // one value in every lane
}

// FP32 area results accepted when 2 u (L P + T) / U, an estimate of the IoU
// rounding error (P: summed edge lengths of the intersection, T: summed
// magnitudes of all shoelace products), is below this (the IoU tolerance is
// 1e-5).
constexpr float kAreaEstMax = 2e-6f;

template <int K>
__device__ __noinline__ void warp_robust(const float* __restrict__ p1, const float* __restrict__ p2, int n1, int n2,
                                         bool refine, FwdOut<K>& o) {
    typedef typename MaskOf<K>::T M;
    constexpr int KK = K * K;
    constexpr int C = 2 * K;
    constexpr int ROUNDS = (2 * KK + 31) / 32;
    constexpr unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float px[K], py[K], qx[K], qy[K];
    load_poly<K>(p1, px, py);
    load_poly<K>(p2, qx, qy);
    const float ox = px[0], oy = py[0];
    float Lf = 0.f;
#pragma unroll
    for (int v = 0; v < K; ++v) {
        Lf = fmaxf(Lf, (v < n1) ? fmaxf(fabsf(px[v] - ox), fabsf(py[v] - oy)) : 0.f);
        Lf = fmaxf(Lf, (v < n2) ? fmaxf(fabsf(qx[v] - ox), fabsf(qy[v] - oy)) : 0.f);
    }
    const float thr32 = kDegenRel * Lf * Lf, route32 = kRouteRel * Lf * Lf;

    // orientation tests: index q < KK is S(i,j), KK <= q < 2KK is T(i,j)
    M posS = 0, negS = 0, posT = 0, negT = 0;
    float vf[ROUNDS];
    bool deg = !(Lf > 0.f);
#pragma unroll
    for (int r = 0; r < ROUNDS; ++r) {
        const int q = lane + 32 * r;
        const bool isT = q >= KK;
        const int rem = isT ? q - KK : q;
        const int i = rem / K, j = rem % K;
        const bool valid = q < 2 * KK && i < n1 && j < n2;
        const int i1 = (i + 1 < n1) ? i + 1 : 0, j1 = (j + 1 < n2) ? j + 1 : 0;
        const float Ax = isT ? sel<K>(px, i) : sel<K>(qx, j), Ay = isT ? sel<K>(py, i) : sel<K>(qy, j);
        const float Bx = isT ? sel<K>(px, i1) : sel<K>(qx, j1), By = isT ? sel<K>(py, i1) : sel<K>(qy, j1);
        const float Px = isT ? sel<K>(qx, j) : sel<K>(px, i), Py = isT ? sel<K>(qy, j) : sel<K>(py, i);
        // FP32 in the local frame first: beyond kRouteRel L^2 its sign is
        // exact (see kRouteRel); only the lanes below take the FP64 test.
        // Everything else stays in FP32 (GB300's FP64 rate is a small
        // fraction of its FP32 rate, and many warps run this at once).
        float v = orient32nc(Ax - ox, Ay - oy, Bx - ox, By - oy, Px - ox, Py - oy);
        bool pos = v > 0.f, neg = v < 0.f;
        // a point equal to an endpoint of the edge has orientation exactly 0,
        // and the uncontracted FP32 form above gives exactly 0 there too
        const bool coinc = (Px == Ax && Py == Ay) || (Px == Bx && Py == By);
        const bool need = refine && valid && !coinc && !(fabsf(v) > route32);
        if (__any_sync(full, need)) {
            if (need) {
                const double v64 = orient64(Ax, Ay, Bx, By, Px, Py);
                pos = v64 > 0.0;
                neg = v64 < 0.0;
                v = (float)v64;
            }
        }
        vf[r] = v;
        deg |= valid && !(fabsf(v) > thr32);
        const unsigned bp = __ballot_sync(full, valid && pos), bn = __ballot_sync(full, valid && neg);
        if constexpr (K == 4) {
            posS = bp & 0xFFFFu;
            negS = bn & 0xFFFFu;
            posT = bp >> 16;
            negT = bn >> 16;
        } else {
            const int sh = 32 * (r & 1);
            if (r < 2) {
                posS |= (M)bp << sh;
                negS |= (M)bn << sh;
            } else {
                posT |= (M)bp << sh;
                negT |= (M)bn << sh;
            }
        }
    }

    constexpr M kRow0 = (M)((1ull << K) - 1);
    M col0 = 0, rows = 0, cols = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) col0 |= (M)1 << (i * K);
#pragma unroll
    for (int i = 0; i < K; ++i) rows |= (i < n1) ? (kRow0 << (i * K)) : (M)0;
#pragma unroll
    for (int j = 0; j < K; ++j) cols |= (j < n2) ? (col0 << j) : (M)0;
    const M V = rows & cols;
    // strict sign change along P1 edge i (rows i, i+1) and along P2 edge j (columns j, j+1)
    const M posSn = ((posS >> K) & ~(kRow0 << (K * (n1 - 1)))) | ((posS & kRow0) << (K * (n1 - 1)));
    const M negSn = ((negS >> K) & ~(kRow0 << (K * (n1 - 1)))) | ((negS & kRow0) << (K * (n1 - 1)));
    const M posTn = ((posT >> 1) & ~(col0 << (n2 - 1))) | ((posT & col0) << (n2 - 1));
    const M negTn = ((negT >> 1) & ~(col0 << (n2 - 1))) | ((negT & col0) << (n2 - 1));
    const M X = ((posS & negSn) | (negS & posSn)) & ((posT & negTn) | (negT & posTn)) & V;
    // inclusive inside tests, exact duplicates of P1 vertices dropped from P2's
    uint32_t in1 = 0, in2 = 0;
    const M nnS = V & ~negS, nnT = V & ~negT;
    const M colsFull = (M)((1ull << n2) - 1);
    M rowsCol = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) rowsCol |= (i < n1) ? ((M)1 << (i * K)) : (M)0;
#pragma unroll
    for (int i = 0; i < K; ++i) {
        in1 |= (i < n1 && ((nnS >> (i * K)) & colsFull) == colsFull) ? (1u << i) : 0u;
        in2 |= (i < n2 && ((nnT >> i) & rowsCol) == rowsCol) ? (1u << i) : 0u;
    }
    bool dup = false;
    if (lane < n2) {
        const float mx_ = sel<K>(qx, lane), my_ = sel<K>(qy, lane);
#pragma unroll
        for (int i = 0; i < K; ++i) dup |= i < n1 && px[i] == mx_ && py[i] == my_;
    }
    in2 &= ~__ballot_sync(full, dup);

    const int c1n = __popc(in1), c2n = __popc(in2), cxn = popc_(X);
    const int m = c1n + c2n + cxn;
    o.nx = 0;
    o.ai = 0.f;
    o.iou = 0.f;
    codes_fill<K>(o.codes, ~0ull);

    // candidate of this lane: a vertex (t = 0) or a crossing a + t (a1 - a)
    const bool live = lane < m && m <= C;
    int ci = 0, cj = 0, kind = 3;
    if (live) {
        if (lane < c1n) {
            kind = 0;
            ci = (int)__fns(in1, 0, lane + 1);
        } else if (lane < c1n + c2n) {
            kind = 1;
            cj = (int)__fns(in2, 0, lane - c1n + 1);
        } else {
            const int cc = lane - c1n - c2n;
            int b;
            if constexpr (K == 4) {
                b = (int)__fns((uint32_t)X, 0, cc + 1);
            } else {
                const uint32_t lo = (uint32_t)X, hi = (uint32_t)(X >> 32);
                const int nlo = __popc(lo);
                b = (cc < nlo) ? (int)__fns(lo, 0, cc + 1) : 32 + (int)__fns(hi, 0, cc - nlo + 1);
            }
            kind = 2;
            ci = b / K;
            cj = b % K;
        }
    }
    const int ci1 = (ci + 1 < n1) ? ci + 1 : 0, cj1 = (cj + 1 < n2) ? cj + 1 : 0;
    // S(i,j), S(i+1,j) and T(i,j), T(i,j+1) from the lanes that computed them
    const int qs[4] = {ci * K + cj, ci1 * K + cj, KK + ci * K + cj, KK + ci * K + cj1};
    float ov[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        ov[f] = 0.f;
#pragma unroll
        for (int r = 0; r < ROUNDS; ++r) {
            const float t = __shfl_sync(full, vf[r], qs[f] & 31);
            ov[f] = ((qs[f] >> 5) == r) ? t : ov[f];
        }
    }
    uint32_t code = 0xFFu;
    float fx0 = 0.f, fy0 = 0.f, fx1 = 0.f, fy1 = 0.f, t = 0.f;
    float gx0 = 0.f, gy0 = 0.f, gx1 = 0.f, gy1 = 0.f; // P2 edge of a crossing
    bool deg2 = false;
    if (kind == 0) {
        code = (uint32_t)ci;
        fx0 = fx1 = sel<K>(px, ci);
        fy0 = fy1 = sel<K>(py, ci);
    } else if (kind == 1) {
        code = 0x40u | (uint32_t)cj;
        fx0 = fx1 = sel<K>(qx, cj);
        fy0 = fy1 = sel<K>(qy, cj);
    } else if (kind == 2) {
        code = 0x80u | ((uint32_t)ci << 3) | (uint32_t)cj;
        fx0 = sel<K>(px, ci);
        fy0 = sel<K>(py, ci);
        fx1 = sel<K>(px, ci1);
        fy1 = sel<K>(py, ci1);
        const float bx0 = sel<K>(qx, cj), by0 = sel<K>(qy, cj), bx1 = sel<K>(qx, cj1), by1 = sel<K>(qy, cj1);
        gx0 = bx0;
        gy0 = by0;
        gx1 = bx1;
        gy1 = by1;
        // the crossing parameters only place a vertex along its edge, so they
        // are FP32 quotients of the orientation values (of opposite signs at
        // a strict crossing, so the differences do not cancel)
        t = ov[0] / (ov[0] - ov[1]);
        const float u = ov[2] / (ov[2] - ov[3]);
        const float rx = fx1 - fx0, ry = fy1 - fy0, sx = bx1 - bx0, sy = by1 - by0;
        const float D = rx * sy - ry * sx;
        deg2 = t <= kDegenRel || t >= 1.0f - kDegenRel || u <= kDegenRel || u >= 1.0f - kDegenRel ||
               D * D <= kDegenRel * kDegenRel * (rx * rx + ry * ry) * (sx * sx + sy * sy);
    }
    deg = __any_sync(full, deg || deg2);
    o.degen = (deg ? 1u : 0u) | (refine ? 2u : 0u);
    if (m > C) {
        o.err |= kDevOverflow;
        o.degen |= 1u;
        return;
    }
    if (m < 3) {
        // empty intersection: the inputs' areas are still reported (the union)
        float s1 = 0.f, s2 = 0.f;
        if (lane < K) {
            const int v = lane, w = (lane + 1 < n1) ? lane + 1 : 0, w2 = (lane + 1 < n2) ? lane + 1 : 0;
            const float X1 = sel<K>(px, v) - ox, Y1 = sel<K>(py, v) - oy, X2 = sel<K>(px, w) - ox, Y2 = sel<K>(py, w) - oy;
            const float U1 = sel<K>(qx, v) - ox, V1 = sel<K>(qy, v) - oy, U2 = sel<K>(qx, w2) - ox, V2 = sel<K>(qy, w2) - oy;
            s1 = (v < n1) ? X1 * Y2 - Y1 * X2 : 0.f;
            s2 = (v < n2) ? U1 * V2 - V1 * U2 : 0.f;
        }
        o.a1 = 0.5f * warp_sum_f(s1);
        o.a2 = 0.5f * warp_sum_f(s2);
        return;
    }
    const float x = (fx0 - ox) + t * (fx1 - fx0), y = (fy0 - oy) + t * (fy1 - fy0);

    // angular order about the centroid, ties by code; rotate to the smallest code
    const float mxf = warp_sum_f(live ? x : 0.f) / (float)m, myf = warp_sum_f(live ? y : 0.f) / (float)m;
    const float key = live ? pseudo_angle(x - mxf, y - myf) : __int_as_float(0x7f800000);
    int rank = 0;
    for (int l = 0; l < m; ++l) {
        const float k2 = __shfl_sync(full, key, l);
        const uint32_t c2 = __shfl_sync(full, code, l);
        rank += (k2 < key || (k2 == key && c2 < code)) ? 1 : 0;
    }
    uint32_t cmin = live ? code : 0xFFFFu;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) cmin = min(cmin, __shfl_xor_sync(full, cmin, off));
    const int src = __ffs(__ballot_sync(full, live && code == cmin)) - 1;
    const int r0 = __shfl_sync(full, rank, src);
    const int slot = (rank - r0 + m) % m;
    unsigned long long w0 = 0, w1 = 0;
    if (live) {
        if (slot < 8) w0 = (unsigned long long)code << (8 * slot);
        else w1 = (unsigned long long)code << (8 * (slot - 8));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        w0 |= __shfl_xor_sync(full, w0, off);
        w1 |= __shfl_xor_sync(full, w1, off);
    }
    const unsigned long long fill0 = (m >= 8) ? 0ull : (~0ull << (8 * m));
    const unsigned long long fill1 = (m >= 16) ? 0ull : (m <= 8 ? ~0ull : (~0ull << (8 * (m - 8))));
    o.codes.w[0] = w0 | fill0;
    if constexpr (K > 4) o.codes.w[1] = w1 | fill1;

    // lane holding the next vertex (slot + 1) of the cycle
    const int target = (slot + 1 == m) ? 0 : slot + 1;
    int nl = 0;
    for (int s2 = 0; s2 < m; ++s2) {
        const unsigned bs = __ballot_sync(full, live && slot == s2);
        nl = (s2 == target) ? __ffs(bs) - 1 : nl;
    }
    const float xn = __shfl_sync(full, x, nl), yn = __shfl_sync(full, y, nl);

    // FP32 areas: the intersection about its centroid, each input about its
    // first vertex, with the magnitudes of their products
    float term = 0.f, mag = 0.f, edge = 0.f;
    if (live) {
        const float ux = x - mxf, uy = y - myf, vx = xn - mxf, vy = yn - myf;
        term = ux * vy - uy * vx;
        mag = fabsf(ux * vy) + fabsf(uy * vx);
        edge = fabsf(xn - x) + fabsf(yn - y);
    }
    float term2 = 0.f, mag2 = 0.f;
    const int v = lane & 7;
    const bool second = lane >= 8 && lane < 16;
    const int nv = second ? n2 : n1;
    const bool on = lane < 16 && v < nv;
    const int wv = (v + 1 < nv) ? v + 1 : 0;
    float xv = 0.f, yv = 0.f, xw = 0.f, yw = 0.f;
#pragma unroll
    for (int m2 = 0; m2 < K; ++m2) {
        xv = (m2 == v) ? (second ? qx[m2] : px[m2]) : xv;
        yv = (m2 == v) ? (second ? qy[m2] : py[m2]) : yv;
        xw = (m2 == wv) ? (second ? qx[m2] : px[m2]) : xw;
        yw = (m2 == wv) ? (second ? qy[m2] : py[m2]) : yw;
    }
    const float bx = second ? qx[0] : px[0], by = second ? qy[0] : py[0];
    if (on) {
        const float Xv = xv - bx, Yv = yv - by, Xw = xw - bx, Yw = yw - by;
        term2 = Xv * Yw - Yv * Xw;
        mag2 = fabsf(Xv * Yw) + fabsf(Yv * Xw);
    }
    const float ai = 0.5f * warp_sum_f(term);
    const float a1 = 0.5f * warp_sum_f(lane < 8 ? term2 : 0.f);
    const float a2 = 0.5f * warp_sum_f(second ? term2 : 0.f);
    const float magsum = warp_sum_f(mag + mag2), perim = warp_sum_f(edge);
    float U = a1 + a2 - ai;
    const float est = 2.f * 5.9604645e-8f * (Lf * 2.f * perim + magsum);
    o.nx = (uint32_t)m;
    o.ai = ai;
    o.a1 = a1;
    o.a2 = a2;
    if (refine && !(est <= kAreaEstMax * U)) {
        // Float-float areas: every vertex placed on its edge in float-float
        // (a crossing's parameter from its two orientations about the P2
        // edge, which have opposite signs at a proper crossing, so their
        // difference does not cancel), the intersection about the
        // candidates' FP32 centroid, the inputs about P1's vertex 0.
        ff X(0.f), Y(0.f);
        if (live) {
            const ff f0x = ff_two_sum(fx0, -ox), f0y = ff_two_sum(fy0, -oy);
            if (kind == 2) {
                // S = orient(g0, g1, f) for both ends of the P1 edge, exactly
                // as float-float from the FP32 inputs
                const ff sx = ff_two_sum(gx1, -gx0), sy = ff_two_sum(gy1, -gy0);
                const ff s0 = sx * ff_two_sum(fy0, -gy0) - sy * ff_two_sum(fx0, -gx0);
                const ff s1 = sx * ff_two_sum(fy1, -gy0) - sy * ff_two_sum(fx1, -gx0);
                const ff tt = s0 / (s0 - s1);
                X = f0x + tt * ff_two_sum(fx1, -fx0);
                Y = f0y + tt * ff_two_sum(fy1, -fy0);
            } else {
                X = f0x;
                Y = f0y;
            }
        }
        // about the FP32 centroid: any origin gives the same area, and one
        // within the polygon keeps the products small
        const ff mx(mxf), my(myf);
        const ff Xn = shfl(full, X, nl), Yn = shfl(full, Y, nl);
        ff tm = live ? (X - mx) * (Yn - my) - (Y - my) * (Xn - mx) : ff(0.f);
        ff t2(0.f);
        if (on) {
            const ff Xv = ff_two_sum(xv, -ox), Yv = ff_two_sum(yv, -oy), Xw = ff_two_sum(xw, -ox),
                     Yw = ff_two_sum(yw, -oy);
            t2 = Xv * Yw - Yv * Xw;
        }
        ff t1 = lane < 8 ? t2 : ff(0.f), t3 = second ? t2 : ff(0.f);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            tm += shfl_xor(full, tm, off);
            t1 += shfl_xor(full, t1, off);
            t3 += shfl_xor(full, t3, off);
        }
        const ff half(0.5f);
        const ff aiF = half * tm, a1F = half * t1, a2F = half * t3;
        o.ai = (float)aiF;
        o.a1 = (float)a1F;
        o.a2 = (float)a2F;
        const ff UF = a1F + a2F - aiF;
        o.iou = (UF > ff(0.f)) ? (float)(aiF / UF) : 0.f;
        return;
    }
    o.iou = (U > 0.f) ? ai / U : 0.f;
}

// ------------------------------------------------------ metrics of the areas
//
// The backward paths take the derivative of the loss with respect to the
// three areas (A_i, A_1, A_2) from a policy object, so the same clip
// adjoint serves the 2D IoU and the 3D IoU.

// 1 / U: in FP32 the approximate reciprocal refined by one Newton step
// (within about 1 ulp, and without the branch of IEEE division; the
// gradients it scales are checked to 1e-3), in float-float its quotient.
__device__ __forceinline__ float recip_adj(float U) {
    const float r = __fdividef(1.0f, U);
    return r * fmaf(-U, r, 2.0f);
}
__device__ __forceinline__ ff recip_adj(ff U) { return ff(1.0f) / U; }

// L = g IoU + e (A_i - A_1 - A_2), IoU = A_i / (A_1 + A_2 - A_i) (paper
// Sec. II-B `iou`); e = 0 except in the GIoU loss, where the term -U / A_h of
// the loss adds it (with the hull area A_h held fixed here).
struct AdjIou {
    float g;
    float e;
    template <typename R>
    __device__ __forceinline__ bool operator()(R ai, R a1, R a2, R& gai, R& ga1, R& ga2) {
        const R U = a1 + a2 - ai;
        if (!(U > (R)0)) return false;
        const R rU = recip_adj(U);
        gai = (R)g * (a1 + a2) * rU * rU + (R)e;
        ga1 = ga2 = -(R)g * ai * rU * rU - (R)e;
        return true;
    }
};

// Vertical extents of a pair of 3D boxes, (z_center, height) each: the
// overlap ov = min(hi1, hi2) - max(lo1, lo2) clamped at 0, and which box's
// ends bound it (P1's at ties).
struct ZPair {
    float h1, h2, ov;
    bool pos, top1, bot1;
};

__device__ __forceinline__ ZPair z_pair(float2 z1, float2 z2) {
    ZPair z;
    const float lo1 = z1.x - 0.5f * z1.y, hi1 = z1.x + 0.5f * z1.y;
    const float lo2 = z2.x - 0.5f * z2.y, hi2 = z2.x + 0.5f * z2.y;
    const float ov = fminf(hi1, hi2) - fmaxf(lo1, lo2);
    z.h1 = z1.y;
    z.h2 = z2.y;
    z.pos = ov > 0.f;
    z.ov = z.pos ? ov : 0.f;
    z.top1 = hi1 <= hi2;
    z.bot1 = lo1 >= lo2;
    return z;
}

// 3D IoU of boxes given as a bird's-eye-view polygon and a vertical extent
// (the rotated 3D IoU of the paper's Sec. IV-A): IoU3 = I / U3 with
// I = A_i ov, U3 = A_1 h_1 + A_2 h_2 - I; 0 when U3 <= 0.
__device__ __forceinline__ float iou3_value(float ai, float a1, float a2, uint32_t nx, const ZPair& z) {
    const float I = (nx >= 3u ? ai : 0.f) * z.ov;
    const float U = a1 * z.h1 + a2 * z.h2 - I;
    return U > 0.f ? I / U : 0.f;
}

// L = g IoU3; records the areas it was given, for dL/d(z, h).
struct AdjIou3 {
    float g;
    ZPair z;
    float ai, a1, a2;
    bool hit;
    template <typename R>
    __device__ __forceinline__ bool operator()(R ai_, R a1_, R a2_, R& gai, R& ga1, R& ga2) {
        const R I = ai_ * (R)z.ov, V1 = a1_ * (R)z.h1, V2 = a2_ * (R)z.h2, U = V1 + V2 - I;
        hit = U > (R)0;
        ai = (float)ai_;
        a1 = (float)a1_;
        a2 = (float)a2_;
        if (!hit) return false;
        const R rU = (R)1 / U;
        const R dI = (V1 + V2) * rU * rU, dV = -I * rU * rU; // dIoU3/dI, dIoU3/dV_k
        gai = (R)g * dI * (R)z.ov;
        ga1 = (R)g * dV * (R)z.h1;
        ga2 = (R)g * dV * (R)z.h2;
        return true;
    }
    // dL/d(z_center, height) of both boxes (zero unless the areas were taken
    // with a positive union): through ov = min(hi1, hi2) - max(lo1, lo2),
    // hi = z + h/2, lo = z - h/2, and V_k = A_k h_k.
    __device__ __forceinline__ void z_grads(float2& gz1, float2& gz2) const {
        gz1 = gz2 = make_float2(0.f, 0.f);
        if (!hit) return;
        const float I = ai * z.ov, V1 = a1 * z.h1, V2 = a2 * z.h2, U = V1 + V2 - I;
        const float rU = 1.f / U;
        const float dI = (V1 + V2) * rU * rU, dV = -I * rU * rU;
        const float gov = z.pos ? g * dI * ai : 0.f;
        const float t1 = z.top1 ? 1.f : 0.f, b1 = z.bot1 ? 1.f : 0.f;
        gz1 = make_float2(gov * (t1 - b1), gov * 0.5f * (t1 + b1) + g * dV * a1);
        gz2 = make_float2(gov * ((1.f - t1) - (1.f - b1)), gov * 0.5f * ((1.f - t1) + (1.f - b1)) + g * dV * a2);
    }
};

// ---------------------------------------------------------------- backward
//
// Main path (bwd_shape): the shape derivative of the area over the clipped
// edge pieces named by the codes.  List path (warp_bwd, one warp per pair):
// the recorded codes rebuild the intersection vertices (crossings as w = a + t ea,
// t = cross(eb, a - b) / cross(ea, eb)), the shoelace adjoint
// dA/dw_k = 1/2 perp(w_{k+1} - w_{k-1}) gives each vertex's gradient, vertex
// codes route it to that vertex and crossing codes through the adjoint of w
// onto the four endpoints of the two edges; in float-float with refinement.

// Warp-cooperative form of the shoelace adjoint, for the pairs the shape
// derivative cannot take: all 32 lanes work on one pair.  Lane k rebuilds
// intersection vertex k from its code (crossings as w = a + t ea in R) and
// takes its neighbours by shuffle; the three areas are shuffle sums; each
// lane's share dA/dw_k = 1/2 perp(w_{k+1} - w_{k-1}) goes to its vertex, or
// through the adjoint of w onto the four endpoints of the crossing's edges,
// by FP32 atomics into the warp's scratch sh[4K] (P1 x, P1 y, P2 x, P2 y);
// lanes s K + v then add the input-area terms and write the gradients.
// codes / nx / adj / counts are the pair's (uniform over the warp); adj maps
// the areas to their adjoints.  Returns device status bits (the same in every
// lane).
template <int K, typename R, typename Adj>
__device__ __noinline__ uint32_t warp_bwd(const float* __restrict__ p1, const float* __restrict__ p2, int n1, int n2,
                                          Adj& adj, uint32_t nx, Codes<K> codes, float* __restrict__ g1,
                                          float* __restrict__ g2, float* __restrict__ sh) {
    constexpr unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    float px[K], py[K], qx[K], qy[K];
    load_poly<K>(p1, px, py);
    load_poly<K>(p2, qx, qy);
    const R ox = (R)px[0], oy = (R)py[0];
    if (lane < 4 * K) sh[lane] = 0.f;
    __syncwarp();
    // fewer than three vertices: an empty intersection (the inputs' areas
    // still take their adjoints)
    const bool live = nx >= 3u && (uint32_t)lane < nx;
    const uint32_t c = live ? code_at<K>(codes, (uint32_t)lane) : 0xFFu;
    const uint32_t kind = c >> 6, lo = c & 7u, ci = (c >> 3) & 7u;
    bool bad = false;
    R wx = 0, wy = 0;
    // crossing data kept for the adjoint
    R eax = 0, eay = 0, ebx = 0, eby = 0, dx = 0, dy = 0, D = 1, t = 0;
    int i1 = 0, j1 = 0;
    if (live) {
        if (kind == 0u) {
            bad = (c & 0x3Fu) >= (uint32_t)n1;
            wx = (R)sel<K>(px, lo) - ox;
            wy = (R)sel<K>(py, lo) - oy;
        } else if (kind == 1u) {
            bad = (c & 0x3Fu) >= (uint32_t)n2;
            wx = (R)sel<K>(qx, lo) - ox;
            wy = (R)sel<K>(qy, lo) - oy;
        } else if (kind == 2u && ci < (uint32_t)n1 && lo < (uint32_t)n2) {
            i1 = (ci + 1u < (uint32_t)n1) ? (int)ci + 1 : 0;
            j1 = (lo + 1u < (uint32_t)n2) ? (int)lo + 1 : 0;
            const R ax = (R)sel<K>(px, ci) - ox, ay = (R)sel<K>(py, ci) - oy;
            const R bx = (R)sel<K>(qx, lo) - ox, by = (R)sel<K>(qy, lo) - oy;
            eax = ((R)sel<K>(px, i1) - ox) - ax;
            eay = ((R)sel<K>(py, i1) - oy) - ay;
            ebx = ((R)sel<K>(qx, j1) - ox) - bx;
            eby = ((R)sel<K>(qy, j1) - oy) - by;
            dx = ax - bx;
            dy = ay - by;
            D = eax * eby - eay * ebx;
            const R S = ebx * dy - eby * dx;
            bad = !(D != (R)0);
            t = bad ? (R)0 : S / D;
            wx = ax + t * eax;
            wy = ay + t * eay;
        } else {
            bad = true;
        }
    }
    const uint32_t err = __any_sync(full, bad) ? kDevBadFlags : 0u;
    const int nxt = (lane + 1 < (int)nx) ? lane + 1 : 0, prv = (lane == 0) ? (int)nx - 1 : lane - 1;
    const R wxn = shfl(full, wx, nxt), wyn = shfl(full, wy, nxt);
    const R wxp = shfl(full, wx, prv < 0 ? 0 : prv), wyp = shfl(full, wy, prv < 0 ? 0 : prv);
    R twoA = live ? wx * wyn - wy * wxn : (R)0;
    // input areas: lane v (P1) and lane K + v (P2) hold vertex v
    const int side = (lane >= K && lane < 2 * K) ? 1 : 0;
    const int v = lane - side * K;
    const int nv = side ? n2 : n1;
    const bool onv = lane < 2 * K && v < nv;
    const int vn = (v + 1 < nv) ? v + 1 : 0, vp = (v == 0) ? nv - 1 : v - 1;
    R xv = 0, yv = 0, xn = 0, yn = 0, xp = 0, yp = 0;
#pragma unroll
    for (int m = 0; m < K; ++m) {
        const float fx = side ? qx[m] : px[m], fy = side ? qy[m] : py[m];
        xv = (m == v) ? (R)fx - ox : xv;
        yv = (m == v) ? (R)fy - oy : yv;
        xn = (m == vn) ? (R)fx - ox : xn;
        yn = (m == vn) ? (R)fy - oy : yn;
        xp = (m == vp) ? (R)fx - ox : xp;
        yp = (m == vp) ? (R)fy - oy : yp;
    }
    R aterm = onv ? xv * yn - yv * xn : (R)0;
    R s1 = (lane < K) ? aterm : (R)0, s2 = side ? aterm : (R)0;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        twoA += shfl_xor(full, twoA, off);
        s1 += shfl_xor(full, s1, off);
        s2 += shfl_xor(full, s2, off);
    }
    twoA = shfl(full, twoA, 0);
    s1 = shfl(full, s1, 0);
    s2 = shfl(full, s2, 0);
    const R a1 = (R)0.5 * s1, a2 = (R)0.5 * s2, ai = (R)0.5 * twoA;
    R gai = 0, ga1 = 0, ga2 = 0;
    const bool ok = err == 0u && adj(ai, a1, a2, gai, ga1, ga2);
    const R gas = side ? ga2 : ga1;
    if (ok && live) {
        const R gwx = (R)0.5 * gai * (wyn - wyp), gwy = (R)0.5 * gai * (wxp - wxn);
        if (kind == 0u) {
            atomicAdd(sh + lo, (float)gwx);
            atomicAdd(sh + K + lo, (float)gwy);
        } else if (kind == 1u) {
            atomicAdd(sh + 2 * K + lo, (float)gwx);
            atomicAdd(sh + 3 * K + lo, (float)gwy);
        } else {
            // w = a + t ea, t = S / D, S = cross(eb, a - b), D = cross(ea, eb)
            const R gt = gwx * eax + gwy * eay;
            const R gS = gt / D, gD = -gt * t / D;
            const R geax = t * gwx + gD * eby, geay = t * gwy - gD * ebx;
            const R gebx = gS * dy - gD * eay, geby = -gS * dx + gD * eax;
            const R gdx = -gS * eby, gdy = gS * ebx;
            atomicAdd(sh + ci, (float)(gwx + gdx - geax));
            atomicAdd(sh + K + ci, (float)(gwy + gdy - geay));
            atomicAdd(sh + i1, (float)geax);
            atomicAdd(sh + K + i1, (float)geay);
            atomicAdd(sh + 2 * K + lo, (float)(-gdx - gebx));
            atomicAdd(sh + 3 * K + lo, (float)(-gdy - geby));
            atomicAdd(sh + 2 * K + j1, (float)gebx);
            atomicAdd(sh + 3 * K + j1, (float)geby);
        }
    }
    __syncwarp();
    if (lane < 2 * K) {
        float gx = 0.f, gy = 0.f;
        if (ok && onv) {
            gx = sh[2 * side * K + v] + (float)((R)0.5 * gas * (yn - yp));
            gy = sh[(2 * side + 1) * K + v] + (float)((R)0.5 * gas * (xp - xn));
        }
        float* g = side ? g2 : g1;
        reinterpret_cast<float2*>(g)[v] = make_float2(gx, gy);
    }
    __syncwarp();
    return err;
}

// dL/dP1, dL/dP2 from the codes in FP32 by the shape derivative of the
// intersection area: moving a vertex moves its two incident edges, and the
// area changes by the normal motion integrated over the clipped pieces of
// those edges.  For edge a_i -> a_i+1 = a_i + ea_i with outward normal
// n = (ea.y, -ea.x) and clipped piece [t0, t1] (t = S/D at a crossing),
//   dA_i/da_i   += n ((1 - t0)^2 - (1 - t1)^2) / 2,
//   dA_i/da_i+1 += n (t1^2 - t0^2) / 2,
// and the same for P2's edges with u = -T/D; the areas of the inputs are the
// full-edge case [0, 1].  Every index is static.  Returns device status bits,
// or kSlow when the pair must take the shoelace adjoint instead: codes that do
// not describe two convex polygons in general position (edge piece counts
// inconsistent with the inside vertices), or, with refinement, an
// intersection smaller than 1e-5 L^2 (its piece lengths are differences of
// nearby FP32 crossing parameters).
constexpr uint32_t kSlow = 0x80000000u;
constexpr float kTinyArea = 1e-5f;

// Decoding table for quadrilateral codes (K = 4): entry c is what code byte c
// contributes to the masks of bwd_shape: bit v (P1 vertex v), bit 4 + v (P2
// vertex v), bit 8 + 4i + j (crossing of P1 edge i with P2 edge j), bit 24 (a
// code no quadrilateral pair can have).  0xFF (an unused slot) contributes
// nothing.  Generated at compile time; 1 KB, read through L1.
struct CodeLut4 {
    uint32_t e[256];
};
constexpr uint32_t code_entry4(uint32_t c) {
    if (c == 0xFFu) return 0u;
    const uint32_t kind = c >> 6;
    if (kind == 0u) return c < 4u ? (1u << c) : (1u << 24);
    if (kind == 1u) return (c & 0x3Fu) < 4u ? (1u << (4u + (c & 0x3Fu))) : (1u << 24);
    if (kind == 2u) {
        const uint32_t i = (c >> 3) & 7u, j = c & 7u;
        return (i < 4u && j < 4u) ? (1u << (8u + 4u * i + j)) : (1u << 24);
    }
    return 1u << 24;
}
constexpr CodeLut4 make_code_lut4() {
    CodeLut4 L{};
    for (uint32_t c = 0; c < 256u; ++c) L.e[c] = code_entry4(c);
    return L;
}
static __device__ const CodeLut4 g_code_lut4 = make_code_lut4();

template <int K, bool COUNTS, typename Adj>
__device__ __forceinline__ uint32_t bwd_shape(const Geo<K>& g, Adj& adj, uint32_t nx, const Codes<K>& codes,
                                              bool refine, float (&g1x)[K], float (&g1y)[K], float (&g2x)[K],
                                              float (&g2y)[K]) {
    typedef typename MaskOf<K>::T M;
    constexpr int C = 2 * K;
    constexpr M kRow0 = (M)((1ull << K) - 1);
    M col0 = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) col0 |= (M)1 << (i * K);
    const int n1 = g.n1, n2 = g.n2;
    const uint32_t n1m = COUNTS ? (uint32_t)n1 : (uint32_t)K, n2m = COUNTS ? (uint32_t)n2 : (uint32_t)K;
#pragma unroll
    for (int v = 0; v < K; ++v) { g1x[v] = g1y[v] = g2x[v] = g2y[v] = 0.f; }
    if (nx > (uint32_t)C) return kDevBadFlags;
    // fewer than three vertices: an empty intersection (no piece on any edge),
    // taken by the same arithmetic as the other pairs
    const bool empty = nx < 3u;

    // inside vertices and crossings named by the codes
    uint32_t in1 = 0, in2 = 0, other = 0;
    M X = 0;
    if constexpr (K == 4) {
        // slots past nx read as unused (0xFF); one table entry per slot
        const uint64_t live = empty ? 0ull : (nx >= 8u) ? ~0ull : ((1ull << (8u * nx)) - 1ull);
        const uint64_t w = codes.w[0] | ~live;
        const uint32_t lo = (uint32_t)w, hi = (uint32_t)(w >> 32);
        uint32_t acc = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            acc |= __ldg(&g_code_lut4.e[(lo >> (8 * k)) & 0xFFu]);
            acc |= __ldg(&g_code_lut4.e[(hi >> (8 * k)) & 0xFFu]);
        }
        in1 = acc & 15u;
        in2 = (acc >> 4) & 15u;
        X = (M)((acc >> 8) & 0xFFFFu);
        other = acc >> 24;
        if constexpr (COUNTS) {
            // crossings of padded edges
            M valid = 0;
#pragma unroll
            for (int i = 0; i < K; ++i)
#pragma unroll
                for (int j = 0; j < K; ++j) valid |= (i < n1 && j < n2) ? ((M)1 << (i * K + j)) : (M)0;
            other |= (X & ~valid) ? 1u : 0u;
        }
    } else {
#pragma unroll
        for (int k = 0; k < C; ++k) {
            const uint32_t c = code_at<K>(codes, (uint32_t)k);
            const bool live = !empty && (uint32_t)k < nx;
            const uint32_t kind = c >> 6, lo = c & 7u, ci = (c >> 3) & 7u;
            in1 |= (live && kind == 0u) ? (1u << (c & 0x1Fu)) : 0u;
            in2 |= (live && kind == 1u) ? (1u << (c & 0x1Fu)) : 0u;
            X |= (live && kind == 2u) ? ((M)1 << (ci * K + lo)) : (M)0;
            other |= (live && (kind == 3u || (kind == 2u && (ci >= n1m || lo >= n2m)))) ? 1u : 0u;
        }
    }
    if (other || (in1 >> n1m) || (in2 >> n2m)) return kDevBadFlags;
    // edge piece counts must match the inside vertices: no crossing between
    // two inside vertices, one between inside and outside, none or two
    // between two outside vertices; and every code must be distinct
    bool ok = empty || (__popc(in1) + __popc(in2) + popc_(X)) == (int)nx;
    if constexpr (K == 4 && !COUNTS) {
        // The same rule on all eight edges at once, in 4-bit fields: field i
        // of R counts the crossings of P1 edge i (row i of X), field j of C
        // those of P2 edge j (row j of X transposed).  An edge whose ends are
        // inside and outside needs count 1 (s = 1), both inside count 0, both
        // outside count 0 or 2 (n = 1 masks bit 1 of the field).
        const uint32_t x = (uint32_t)X;
        uint32_t xt = x, t = (xt ^ (xt >> 3)) & 0x0A0Au;
        xt ^= t ^ (t << 3);
        t = (xt ^ (xt >> 6)) & 0x00CCu;
        xt ^= t ^ (t << 6);
        auto nib_pop = [](uint32_t v) {
            v = (v & 0x5555u) + ((v >> 1) & 0x5555u);
            return (v & 0x3333u) + ((v >> 2) & 0x3333u);
        };
        auto spread = [](uint32_t m) { return (m | (m << 3) | (m << 6) | (m << 9)) & 0x1111u; };
        const uint32_t in1n = ((in1 >> 1) | (in1 << 3)) & 15u, in2n = ((in2 >> 1) | (in2 << 3)) & 15u;
        const uint32_t da = (nib_pop(x) ^ spread(in1 ^ in1n)) & ~(spread(~(in1 | in1n) & 15u) << 1);
        const uint32_t db = (nib_pop(xt) ^ spread(in2 ^ in2n)) & ~(spread(~(in2 | in2n) & 15u) << 1);
        ok &= (da | db) == 0u;
    } else {
#pragma unroll
        for (int i = 0; i < K; ++i) {
            const bool vi = !COUNTS || i < n1, vj = !COUNTS || i < n2;
            const uint32_t ra = (uint32_t)popc_((X >> (i * K)) & kRow0);
            const uint32_t na = (i + 1 < (int)n1m) ? (uint32_t)(i + 1) : 0u;
            const uint32_t a0 = (in1 >> i) & 1u, a1 = (in1 >> na) & 1u;
            ok &= !vi || ((a0 ^ a1) ? (ra == 1u) : (a0 ? ra == 0u : (ra == 0u || ra == 2u)));
            const uint32_t rb = (uint32_t)popc_((X >> i) & col0);
            const uint32_t nb = (i + 1 < (int)n2m) ? (uint32_t)(i + 1) : 0u;
            const uint32_t b0 = (in2 >> i) & 1u, b1 = (in2 >> nb) & 1u;
            ok &= !vj || ((b0 ^ b1) ? (rb == 1u) : (b0 ? rb == 0u : (rb == 0u || rb == 2u)));
        }
    }
    if (!ok) return kSlow;

    // clipped piece of every edge: [t0, t1] on P1 edges, [u0, u1] on P2 edges.
    // With the piece counts checked above, a P1 edge whose start is inside
    // ends at its only crossing, one whose end is inside starts at its only
    // crossing, and one with two crossings runs from the smaller t to the
    // larger; so min / max over the crossings of the edge give the piece
    // without looking at orientation signs.  Off the crossing set the
    // parameters are NaN, which fminf / fmaxf ignore.  The reductions start at
    // t0 = 1, t1 = 0: a crossing's parameter lies in (0, 1), so the start
    // values do not change the min / max over crossings, and an edge with no
    // piece (no crossing, neither end inside) keeps an empty interval whose
    // length max(t1 - t0, 0) is 0, so every term it would add is 0.
    const float kNaN = __int_as_float(0x7fffffff);
    float t0[K], t1[K], u0[K], u1[K];
#pragma unroll
    for (int v = 0; v < K; ++v) { t0[v] = 1.f; t1[v] = 0.f; u0[v] = 1.f; u1[v] = 0.f; }
    // rows are taken two at a time, so that each column's min / max folds
    // two rows per three-operand instruction
    static_assert(K % 2 == 0, "an even capacity");
    float up[K]; // the previous (even) row's u parameters
    // two P2 edges (j, j + 1) per packed instruction
    ColPair cp[K / 2];
#pragma unroll
    for (int h = 0; h < K / 2; ++h) cp[h] = col_pair<K>(g.bx, g.by, g.ebx, g.eby, h);
#pragma unroll
    for (int i = 0; i < K; ++i) {
        float tr[K]; // row i's parameters, reduced after the row
#pragma unroll
        for (int h = 0; h < K / 2; ++h) {
            const int j = 2 * h;
            Blk2 b;
            if (i == 0) b = blk2<true, false>(0.f, 0.f, g.eax[0], g.eay[0], cp[h]);
            else b = blk2<false, false>(g.ax[i], g.ay[i], g.eax[i], g.eay[i], cp[h]);
            const bool m0 = (X >> (i * K + j)) & 1u, m1 = (X >> (i * K + j + 1)) & 1u;
            const float2 rD = f2(m0 ? __fdividef(1.0f, b.D.x) : kNaN, m1 ? __fdividef(1.0f, b.D.y) : kNaN);
            const float2 u = mul2(b.nT, rD);
            const float2 t = mul2(b.S, rD);
            tr[j] = t.x;
            tr[j + 1] = t.y;
            if (i & 1) {
                u0[j] = fmin3(u0[j], up[j], u.x);
                u1[j] = fmax3(u1[j], up[j], u.x);
                u0[j + 1] = fmin3(u0[j + 1], up[j + 1], u.y);
                u1[j + 1] = fmax3(u1[j + 1], up[j + 1], u.y);
            } else {
                up[j] = u.x;
                up[j + 1] = u.y;
            }
        }
#pragma unroll
        for (int j = 0; j + 1 < K; j += 2) {
            t0[i] = fmin3(t0[i], tr[j], tr[j + 1]);
            t1[i] = fmax3(t1[i], tr[j], tr[j + 1]);
        }
    }
    // an inside start vertex opens its edge's piece at 0, an inside end
    // vertex closes it at 1
    const float L = pair_scale<K, COUNTS>(g);
    float dta[K], dtb[K]; // piece lengths
#pragma unroll
    for (int v = 0; v < K; ++v) {
        const uint32_t na = (v + 1 < (int)n1m) ? (uint32_t)(v + 1) : 0u, nb = (v + 1 < (int)n2m) ? (uint32_t)(v + 1) : 0u;
        t0[v] = ((in1 >> v) & 1u) ? 0.f : t0[v];
        t1[v] = ((in1 >> na) & 1u) ? 1.f : t1[v];
        u0[v] = ((in2 >> v) & 1u) ? 0.f : u0[v];
        u1[v] = ((in2 >> nb) & 1u) ? 1.f : u1[v];
        dta[v] = fmaxf(t1[v] - t0[v], 0.f);
        dtb[v] = fmaxf(u1[v] - u0[v], 0.f);
    }
    float twoA = 0.f, s1 = 0.f, s2 = 0.f;
#pragma unroll
    for (int v = 0; v < K; ++v) {
        const float c1 = g.ax[v] * g.eay[v] - g.ay[v] * g.eax[v];
        const float c2 = g.bx[v] * g.eby[v] - g.by[v] * g.ebx[v];
        s1 += (!COUNTS || v < n1) ? c1 : 0.f;
        s2 += (!COUNTS || v < n2) ? c2 : 0.f;
        twoA = fmaf(dta[v], c1, twoA);
        twoA = fmaf(dtb[v], c2, twoA);
    }
    const float a1 = 0.5f * s1, a2 = 0.5f * s2, ai = 0.5f * twoA;
    if (refine && !empty && ai < kTinyArea * L * L) return kSlow;
    float gai, ga1, ga2;
    if (!adj(ai, a1, a2, gai, ga1, ga2)) return 0u;
    const float h1 = 0.5f * ga1, h2 = 0.5f * ga2, hg = 0.5f * gai;
    // Start / end weights of every edge: the piece [t0, t1] moves the start
    // vertex by ((1 - t0)^2 - (1 - t1)^2) / 2 = (t1 - t0)(2 - t0 - t1) / 2 and
    // the end vertex by (t1^2 - t0^2) / 2 = (t1 - t0)(t1 + t0) / 2 (times the
    // edge normal), plus the full edge of the input's own area.  Vertex v
    // takes the start of edge v and the end of edge v - 1.
    float sx1[K], sy1[K], ex1[K], ey1[K], sx2[K], sy2[K], ex2[K], ey2[K];
#pragma unroll
    for (int v = 0; v < K; ++v) {
        const float da = hg * dta[v], sa = t1[v] + t0[v];
        const float db = hg * dtb[v], sb = u1[v] + u0[v];
        const float wsa = fmaf(da, 2.f - sa, h1), wea = fmaf(da, sa, h1);
        const float wsb = fmaf(db, 2.f - sb, h2), web = fmaf(db, sb, h2);
        sx1[v] = wsa * g.eay[v];
        sy1[v] = -wsa * g.eax[v];
        ex1[v] = wea * g.eay[v];
        ey1[v] = -wea * g.eax[v];
        sx2[v] = wsb * g.eby[v];
        sy2[v] = -wsb * g.ebx[v];
        ex2[v] = web * g.eby[v];
        ey2[v] = -web * g.ebx[v];
    }
    float lx1 = ex1[K - 1], ly1 = ey1[K - 1], lx2 = ex2[K - 1], ly2 = ey2[K - 1];
    if constexpr (COUNTS) {
        lx1 = sel<K>(ex1, (uint32_t)(n1 - 1));
        ly1 = sel<K>(ey1, (uint32_t)(n1 - 1));
        lx2 = sel<K>(ex2, (uint32_t)(n2 - 1));
        ly2 = sel<K>(ey2, (uint32_t)(n2 - 1));
    }
#pragma unroll
    for (int v = 0; v < K; ++v) {
        const bool v1 = !COUNTS || v < n1, v2 = !COUNTS || v < n2;
        g1x[v] = v1 ? sx1[v] + (v ? ex1[v - 1] : lx1) : 0.f;
        g1y[v] = v1 ? sy1[v] + (v ? ey1[v - 1] : ly1) : 0.f;
        g2x[v] = v2 ? sx2[v] + (v ? ex2[v - 1] : lx2) : 0.f;
        g2y[v] = v2 ? sy2[v] + (v ? ey2[v - 1] : ly2) : 0.f;
    }
    return 0u;
}

} // namespace dgal
