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
//   * the area is the shoelace sum grouped by edge: each clipped edge piece
//     contributes cross(start, end), its endpoints being polygon vertices or
//     crossing points a_i + t ea_i (t = S/D, D = cross(ea_i, eb_j)), so no
//     vertex ordering is needed for it.
//   Near-degenerate pairs, and pairs whose walk does not close, take a
//   separate robust path (candidate gathering and an angular sort; with
//   refinement, FP64 orientation tests, crossing parameters and areas).
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

// device status bits (mirror include/dgal.h)
constexpr uint32_t kDevBadCount = 0x1u;
constexpr uint32_t kDevOverflow = 0x2u;
constexpr uint32_t kDevBadFlags = 0x4u;
constexpr uint32_t kDevBadOffsets = 0x8u;

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

// Value at dynamic index idx of a register array (select chain, no local memory).
template <int K> __device__ __forceinline__ float sel(const float (&a)[K], uint32_t idx) {
    float r = a[0];
#pragma unroll
    for (int m = 1; m < K; ++m) r = (idx == (uint32_t)m) ? a[m] : r;
    return r;
}

template <int K> __device__ __forceinline__ void add_at(float (&a)[K], uint32_t idx, float v) {
#pragma unroll
    for (int m = 0; m < K; ++m) a[m] += (idx == (uint32_t)m) ? v : 0.0f;
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
        g.ax[v] = px[v] - ox;
        g.ay[v] = py[v] - oy;
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
#pragma unroll
    for (int v = 0; v < K; ++v) {
        float la = fmaxf(fabsf(g.ax[v]), fabsf(g.ay[v]));
        float lb = fmaxf(fabsf(g.bx[v]), fabsf(g.by[v]));
        L = fmaxf(L, (!COUNTS || v < g.n1) ? la : 0.f);
        L = fmaxf(L, (!COUNTS || v < g.n2) ? lb : 0.f);
    }
    return L;
}

// ------------------------------------------------------------ generic path

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

// Returns false when the pair must take the robust path: some orientation is
// within the near-degenerate threshold (|orient| <= 1e-5 L^2), or the sign
// pattern is not that of two convex polygons in general position.  While every
// |orient| exceeds that threshold (which is far above the FP32 rounding of the
// local-frame values), every sign is exact, so the inside tests, crossings and
// the vertex order are exactly those of the FP64 definition.  On success fills
// o.codes, o.nx and o.ai.
template <int K, bool COUNTS> __device__ __forceinline__ bool fwd_generic(const Geo<K>& g, FwdOut<K>& o) {
    typedef typename MaskOf<K>::T M;
    typedef typename SeqOf<K>::T Sq;
    constexpr int KK = K * K;
    constexpr int C = 2 * K;
    constexpr M kRow0 = (M)((1ull << K) - 1);
    M col0 = 0;
#pragma unroll
    for (int i = 0; i < K; ++i) col0 |= (M)1 << (i * K);
    const int n1 = g.n1, n2 = g.n2;

    const float L = pair_scale<K, COUNTS>(g);
    const float thr = kDegenRel * L * L;

    // Orientation values: S(i,j) = orient(b_j, b_j+1, a_i), T(i,j) =
    // orient(a_i, a_i+1, b_j).  Kept for K = 4, recomputed for K = 8.
    constexpr bool KEEP = (K <= 4);
    float Sv[KEEP ? KK : 1];
    M neg_s = 0, neg_t = 0;
    float minabs = __int_as_float(0x7f800000);
#pragma unroll
    for (int i = 0; i < K; ++i) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const float dx = g.ax[i] - g.bx[j], dy = g.ay[i] - g.by[j];
            const float s = g.ebx[j] * dy - g.eby[j] * dx;
            const float t = g.eay[i] * dx - g.eax[i] * dy;
            if constexpr (KEEP) Sv[i * K + j] = s;
            const bool valid = !COUNTS || (i < n1 && j < n2);
            minabs = fminf(minabs, valid ? fminf(fabsf(s), fabsf(t)) : __int_as_float(0x7f800000));
            neg_s |= (M)(__float_as_uint(s) >> 31) << (i * K + j);
            neg_t |= (M)(__float_as_uint(t) >> 31) << (i * K + j);
        }
    }
    if (!(L > 0.f) || !(minabs > thr)) return false;

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
    {
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

    const uint32_t n2m = COUNTS ? (uint32_t)n2 : (uint32_t)K;
    // Area: the shoelace of the intersection grouped by edge, i.e. the sum over
    // clipped edge pieces of cross(start, end).  A piece of P1 edge i runs from
    // a_i (if inside) or its entry crossing to a_{i+1} (if inside) or its exit
    // crossing; likewise for P2.  Each crossing point is computed once, as
    // a_i + t ea_i with t = S/D, D = cross(ea_i, eb_j), and closes one P1 piece
    // and one P2 piece, so rounding of t moves a vertex along the boundary and
    // does not open a gap between the two pieces.
    float sAx[K], sAy[K], eAx[K], eAy[K], sBx[K], sBy[K], eBx[K], eBy[K];
#pragma unroll
    for (int v = 0; v < K; ++v) {
        sAx[v] = g.ax[v];
        sAy[v] = g.ay[v];
        eAx[v] = g.ax[v] + g.eax[v];
        eAy[v] = g.ay[v] + g.eay[v];
        sBx[v] = g.bx[v];
        sBy[v] = g.by[v];
        eBx[v] = g.bx[v] + g.ebx[v];
        eBy[v] = g.by[v] + g.eby[v];
    }
#pragma unroll
    for (int i = 0; i < K; ++i) {
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int bit = i * K + j;
            float S;
            if constexpr (KEEP) {
                S = Sv[bit];
            } else {
                const float dx = g.ax[i] - g.bx[j], dy = g.ay[i] - g.by[j];
                S = g.ebx[j] * dy - g.eby[j] * dx;
            }
            const float D = g.eax[i] * g.eby[j] - g.eay[i] * g.ebx[j];
            const float t = __fdividef(S, D);
            const float wx = g.ax[i] + t * g.eax[i], wy = g.ay[i] + t * g.eay[i];
            const bool xb = (X >> bit) & 1u;
            const bool en = xb && ((entry1 >> bit) & 1u);
            const bool ex = xb && !((entry1 >> bit) & 1u);
            sAx[i] = en ? wx : sAx[i];
            sAy[i] = en ? wy : sAy[i];
            eBx[j] = en ? wx : eBx[j];
            eBy[j] = en ? wy : eBy[j];
            eAx[i] = ex ? wx : eAx[i];
            eAy[i] = ex ? wy : eAy[i];
            sBx[j] = ex ? wx : sBx[j];
            sBy[j] = ex ? wy : sBy[j];
        }
    }
    float twoA = 0.f;
#pragma unroll
    for (int v = 0; v < K; ++v) {
        const bool hasA = ((in1 >> v) & 1u) || (((entry1 >> (v * K)) & kRow0) != 0);
        const bool hasB = ((in2 >> v) & 1u) || (((exit1 >> v) & col0) != 0);
        twoA += hasA ? sAx[v] * eAy[v] - sAy[v] * eAx[v] : 0.f;
        twoA += hasB ? sBx[v] * eBy[v] - sBy[v] * eBx[v] : 0.f;
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
    const uint32_t jmin = (uint32_t)(__ffs(in2 | 0x100u) - 1);
    const uint32_t fullq = (1u << n2m) - 1u;
    Sq seq = 0;
    uint32_t pos = 0, p0 = 0, qmask = 0;
    bool bad = false;
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

// Shoelace of an ordered point list relative to its first point (double).
__device__ __forceinline__ double shoelace64(const double* x, const double* y, int m) {
    double s = 0.0;
    for (int k = 1; k + 1 < m; ++k)
        s += __dsub_rn(__dmul_rn(x[k] - x[0], y[k + 1] - y[0]), __dmul_rn(y[k] - y[0], x[k + 1] - x[0]));
    return 0.5 * s;
}

// Candidate gathering with the inclusive/strict rules, angular order, shoelace.
// Reloads the raw float inputs so FP64 tests see the unrounded values.  With
// refinement on, a near-degenerate pair takes its orientation signs, crossing
// parameters and shoelace determinants in FP64 (the areas of slivers are
// ill-conditioned in FP32) and its IoU is formed in FP64.
template <int K>
__device__ __noinline__ void fwd_robust(const float* __restrict__ p1, const float* __restrict__ p2, int n1, int n2,
                                        bool refine, FwdOut<K>& o) {
    constexpr int C = 2 * K;
    float px[K], py[K], qx[K], qy[K];
    load_poly<K>(p1, px, py);
    load_poly<K>(p2, qx, qy);
    const float ox = px[0], oy = py[0];
    float ax[K], ay[K], bx[K], by[K];
    float L = 0.f;
    for (int v = 0; v < K; ++v) {
        ax[v] = px[v] - ox;
        ay[v] = py[v] - oy;
        bx[v] = qx[v] - ox;
        by[v] = qy[v] - oy;
        if (v < n1) L = fmaxf(L, fmaxf(fabsf(ax[v]), fabsf(ay[v])));
        if (v < n2) L = fmaxf(L, fmaxf(fabsf(bx[v]), fabsf(by[v])));
    }
    const float thr = kDegenRel * L * L;

    // classifier on FP32 local values
    bool degen = !(L > 0.f);
    signed char sS[K * K], sT[K * K]; // signs: S(i,j) of a_i vs edge j, T(i,j) of b_j vs edge i
    float Sf[K * K], Tf[K * K];
    for (int i = 0; i < n1; ++i) {
        const int i1 = (i + 1 < n1) ? i + 1 : 0;
        for (int j = 0; j < n2; ++j) {
            const int j1 = (j + 1 < n2) ? j + 1 : 0;
            float s = orient32nc(bx[j], by[j], bx[j1], by[j1], ax[i], ay[i]);
            float t = orient32nc(ax[i], ay[i], ax[i1], ay[i1], bx[j], by[j]);
            Sf[i * K + j] = s;
            Tf[i * K + j] = t;
            degen |= (fabsf(s) <= thr) || (fabsf(t) <= thr);
        }
    }
    for (int i = 0; i < n1; ++i) {
        const int i1 = (i + 1 < n1) ? i + 1 : 0;
        for (int j = 0; j < n2; ++j) {
            const int j1 = (j + 1 < n2) ? j + 1 : 0;
            float Sa = Sf[i * K + j], Sb = Sf[i1 * K + j], Ta = Tf[i * K + j], Tb = Tf[i * K + j1];
            bool cross = ((Sa > 0.f && Sb < 0.f) || (Sa < 0.f && Sb > 0.f)) &&
                         ((Ta > 0.f && Tb < 0.f) || (Ta < 0.f && Tb > 0.f));
            if (cross) {
                float as = fabsf(Sa), bs = fabsf(Sb), at = fabsf(Ta), bt = fabsf(Tb);
                degen |= fminf(as, bs) <= kDegenRel * (as + bs);
                degen |= fminf(at, bt) <= kDegenRel * (at + bt);
                float eax = ax[i1] - ax[i], eay = ay[i1] - ay[i];
                float ebx = bx[j1] - bx[j], eby = by[j1] - by[j];
                float D = eax * eby - eay * ebx;
                float r2 = eax * eax + eay * eay, s2 = ebx * ebx + eby * eby;
                degen |= D * D <= (kDegenRel * kDegenRel) * r2 * s2;
            }
        }
    }
    const bool use64 = refine && degen;

    // signs (FP64 from the raw inputs when refining)
    for (int i = 0; i < n1; ++i) {
        const int i1 = (i + 1 < n1) ? i + 1 : 0;
        for (int j = 0; j < n2; ++j) {
            const int j1 = (j + 1 < n2) ? j + 1 : 0;
            if (use64) {
                double s = orient64(qx[j], qy[j], qx[j1], qy[j1], px[i], py[i]);
                double t = orient64(px[i], py[i], px[i1], py[i1], qx[j], qy[j]);
                sS[i * K + j] = (s > 0.0) - (s < 0.0);
                sT[i * K + j] = (t > 0.0) - (t < 0.0);
            } else {
                float s = Sf[i * K + j], t = Tf[i * K + j];
                sS[i * K + j] = (s > 0.f) - (s < 0.f);
                sT[i * K + j] = (t > 0.f) - (t < 0.f);
            }
        }
    }

    // candidates, relative to P1's vertex 0 (exact in double for float inputs)
    double cx[C], cy[C];
    float key[C];
    uint32_t cc[C];
    int m = 0;
    bool overflow = false;
    // P1 vertices inside-or-on P2
    for (int i = 0; i < n1; ++i) {
        bool in = true;
        for (int j = 0; j < n2; ++j) in &= sS[i * K + j] >= 0;
        if (in) {
            if (m < C) {
                cx[m] = (double)px[i] - (double)ox;
                cy[m] = (double)py[i] - (double)oy;
                cc[m] = (uint32_t)i;
                ++m;
            } else overflow = true;
        }
    }
    // P2 vertices inside-or-on P1, except exact copies of P1 vertices
    for (int j = 0; j < n2; ++j) {
        bool in = true, dup = false;
        for (int i = 0; i < n1; ++i) {
            in &= sT[i * K + j] >= 0;
            dup |= (qx[j] == px[i]) && (qy[j] == py[i]);
        }
        if (in && !dup) {
            if (m < C) {
                cx[m] = (double)qx[j] - (double)ox;
                cy[m] = (double)qy[j] - (double)oy;
                cc[m] = 0x40u | (uint32_t)j;
                ++m;
            } else overflow = true;
        }
    }
    // proper crossings
    for (int i = 0; i < n1; ++i) {
        const int i1 = (i + 1 < n1) ? i + 1 : 0;
        for (int j = 0; j < n2; ++j) {
            const int j1 = (j + 1 < n2) ? j + 1 : 0;
            int sa = sS[i * K + j], sb = sS[i1 * K + j], ta = sT[i * K + j], tb = sT[i * K + j1];
            if (sa * sb < 0 && ta * tb < 0) {
                double x, y;
                if (use64) {
                    double Sa = orient64(qx[j], qy[j], qx[j1], qy[j1], px[i], py[i]);
                    double Sb = orient64(qx[j], qy[j], qx[j1], qy[j1], px[i1], py[i1]);
                    double t = Sa / (Sa - Sb);
                    x = ((double)px[i] - (double)ox) + t * ((double)px[i1] - (double)px[i]);
                    y = ((double)py[i] - (double)oy) + t * ((double)py[i1] - (double)py[i]);
                } else {
                    float Sa = Sf[i * K + j], Sb = Sf[i1 * K + j];
                    float t = Sa / (Sa - Sb);
                    x = (double)(ax[i] + t * (ax[i1] - ax[i]));
                    y = (double)(ay[i] + t * (ay[i1] - ay[i]));
                }
                if (m < C) {
                    cx[m] = x;
                    cy[m] = y;
                    cc[m] = 0x80u | ((uint32_t)i << 3) | (uint32_t)j;
                    ++m;
                } else {
                    overflow = true;
                }
            }
        }
    }
    o.degen = (degen ? 1u : 0u) | (use64 ? 2u : 0u);
    o.nx = 0;
    o.ai = 0.f;
    o.iou = 0.f;
    codes_fill<K>(o.codes, ~0ull);
    if (overflow) {
        o.err |= kDevOverflow;
        o.degen |= 1u;
        return;
    }
    if (m < 3) return;

    double mx = 0.0, my = 0.0;
    for (int k = 0; k < m; ++k) { mx += cx[k]; my += cy[k]; }
    mx /= (double)m;
    my /= (double)m;
    for (int k = 0; k < m; ++k) key[k] = pseudo_angle((float)(cx[k] - mx), (float)(cy[k] - my));
    for (int k = 1; k < m; ++k) {
        double kx = cx[k], ky = cy[k];
        float kk = key[k];
        uint32_t kc = cc[k];
        int l = k - 1;
        while (l >= 0 && (key[l] > kk || (key[l] == kk && cc[l] > kc))) {
            cx[l + 1] = cx[l]; cy[l + 1] = cy[l]; key[l + 1] = key[l]; cc[l + 1] = cc[l];
            --l;
        }
        cx[l + 1] = kx; cy[l + 1] = ky; key[l + 1] = kk; cc[l + 1] = kc;
    }
    int s0 = 0;
    for (int k = 1; k < m; ++k) s0 = (cc[k] < cc[s0]) ? k : s0;
    double wx[C], wy[C];
    for (int k = 0; k < m; ++k) {
        const int a = (s0 + k) % m;
        code_put<K>(o.codes, (uint32_t)k, cc[a]);
        wx[k] = cx[a];
        wy[k] = cy[a];
    }
    o.nx = (uint32_t)m;
    if (use64) {
        double sx1[K], sy1[K], sx2[K], sy2[K];
        for (int v = 0; v < n1; ++v) { sx1[v] = px[v]; sy1[v] = py[v]; }
        for (int v = 0; v < n2; ++v) { sx2[v] = qx[v]; sy2[v] = qy[v]; }
        const double ai = shoelace64(wx, wy, m);
        const double a1 = shoelace64(sx1, sy1, n1), a2 = shoelace64(sx2, sy2, n2);
        const double U = a1 + a2 - ai;
        o.ai = (float)ai;
        o.a1 = (float)a1;
        o.a2 = (float)a2;
        o.iou = (U > 0.0) ? (float)(ai / U) : 0.f;
    } else {
        float twoA = 0.f;
        for (int k = 0; k < m; ++k) {
            const int b = (k + 1 < m) ? k + 1 : 0;
            twoA += (float)wx[k] * (float)wy[b] - (float)wy[k] * (float)wx[b];
        }
        o.ai = 0.5f * twoA;
        const float U = o.a1 + o.a2 - o.ai;
        o.iou = (U > 0.f) ? o.ai / U : 0.f;
    }
}

// Full forward for one pair whose polygons are already in registers; the raw
// pointers (this pair's polygons) are only read again by the robust path.
template <int K, bool COUNTS>
__device__ __forceinline__ void fwd_loaded(const float (&px)[K], const float (&py)[K], const float (&qx)[K],
                                           const float (&qy)[K], const float* __restrict__ p1,
                                           const float* __restrict__ p2, int n1, int n2, uint32_t flags, Geo<K>& g,
                                           FwdOut<K>& o) {
    make_geo<K, COUNTS>(px, py, qx, qy, n1, n2, g);
    o.err = 0;
    o.degen = 0;
    input_areas<K, COUNTS>(g, o.a1, o.a2);
    if (fwd_generic<K, COUNTS>(g, o)) {
        const float U = o.a1 + o.a2 - o.ai;
        o.iou = (o.nx >= 3u && U > 0.f) ? o.ai / U : 0.f;
    } else {
        fwd_robust<K>(p1, p2, g.n1, g.n2, (flags & kFlagRefine) && !(flags & kFlagPlain), o);
    }
}

template <int K, bool COUNTS>
__device__ __forceinline__ void fwd_pair(const float* __restrict__ p1, const float* __restrict__ p2, int n1, int n2,
                                         uint32_t flags, Geo<K>& g, FwdOut<K>& o) {
    float px[K], py[K], qx[K], qy[K];
    load_poly<K>(p1, px, py);
    load_poly<K>(p2, qx, qy);
    fwd_loaded<K, COUNTS>(px, py, qx, qy, p1, p2, n1, n2, flags, g, o);
}


// ---------------------------------------------------------------- backward
//
// The recorded codes rebuild the intersection vertices (crossings as
// w = a + t ea, t = cross(eb, a - b) / cross(ea, eb), each computed once), the
// shoelace adjoint dA/dw_k = 1/2 perp(w_{k+1} - w_{k-1}) gives each vertex's
// gradient, vertex codes route it to that vertex and crossing codes through
// the adjoint of w onto the four endpoints of the two edges.  Intersections
// smaller than 1e-6 L^2 are redone in FP64 when refinement is on: their
// vertices are too close together for differences of FP32 local coordinates.

// Shoelace adjoint over the recorded vertex sequence in scalar type R, from the
// raw inputs: vertex codes route straight to that vertex, crossing codes go
// through w = a + t ea, t = cross(eb, a - b) / cross(ea, eb).
template <int K, typename R>
__device__ __noinline__ uint32_t bwd_shoelace(const float* __restrict__ p1, const float* __restrict__ p2, int n1,
                                              int n2, float grad, uint32_t nx, Codes<K> codes, float* __restrict__ g1,
                                              float* __restrict__ g2) {
    constexpr int C = 2 * K;
    float px[K], py[K], qx[K], qy[K];
    load_poly<K>(p1, px, py);
    load_poly<K>(p2, qx, qy);
    R ax[K], ay[K], bx[K], by[K], gax[K], gay[K], gbx[K], gby[K];
    for (int v = 0; v < K; ++v) {
        ax[v] = (R)px[v] - (R)px[0];
        ay[v] = (R)py[v] - (R)py[0];
        bx[v] = (R)qx[v] - (R)px[0];
        by[v] = (R)qy[v] - (R)py[0];
        gax[v] = gay[v] = gbx[v] = gby[v] = (R)0;
    }
    R wx[C], wy[C];
    uint32_t err = 0;
    for (uint32_t k = 0; k < nx; ++k) {
        const uint32_t c = code_at<K>(codes, k);
        const uint32_t kind = c >> 6, lo = c & 7u, ci = (c >> 3) & 7u;
        if (kind == 0u && (c & 0x3Fu) < (uint32_t)n1) {
            wx[k] = ax[lo];
            wy[k] = ay[lo];
        } else if (kind == 1u && (c & 0x3Fu) < (uint32_t)n2) {
            wx[k] = bx[lo];
            wy[k] = by[lo];
        } else if (kind == 2u && ci < (uint32_t)n1 && lo < (uint32_t)n2) {
            const int i1 = (ci + 1u < (uint32_t)n1) ? ci + 1 : 0, j1 = (lo + 1u < (uint32_t)n2) ? lo + 1 : 0;
            const R eax = ax[i1] - ax[ci], eay = ay[i1] - ay[ci], ebx = bx[j1] - bx[lo], eby = by[j1] - by[lo];
            const R D = eax * eby - eay * ebx;
            const R S = ebx * (ay[ci] - by[lo]) - eby * (ax[ci] - bx[lo]);
            if (!(D != (R)0)) { err = kDevBadFlags; break; }
            const R t = S / D;
            wx[k] = ax[ci] + t * eax;
            wy[k] = ay[ci] + t * eay;
        } else {
            err = kDevBadFlags;
            break;
        }
    }
    R a1 = 0, a2 = 0, twoA = 0;
    for (int v = 0; v < n1; ++v) { const int w = (v + 1 < n1) ? v + 1 : 0; a1 += ax[v] * ay[w] - ay[v] * ax[w]; }
    for (int v = 0; v < n2; ++v) { const int w = (v + 1 < n2) ? v + 1 : 0; a2 += bx[v] * by[w] - by[v] * bx[w]; }
    for (uint32_t k = 0; err == 0u && k < nx; ++k) {
        const uint32_t w = (k + 1 < nx) ? k + 1 : 0;
        twoA += wx[k] * wy[w] - wy[k] * wx[w];
    }
    a1 *= (R)0.5;
    a2 *= (R)0.5;
    const R ai = (R)0.5 * twoA, U = a1 + a2 - ai;
    if (err == 0u && U > (R)0) {
        const R gai = (R)grad * (a1 + a2) / (U * U);
        const R ga12 = -(R)grad * ai / (U * U);
        for (uint32_t k = 0; k < nx; ++k) {
            const uint32_t kp = (k == 0) ? nx - 1 : k - 1, kn = (k + 1 < nx) ? k + 1 : 0;
            const R gwx = (R)0.5 * gai * (wy[kn] - wy[kp]);
            const R gwy = (R)0.5 * gai * (wx[kp] - wx[kn]);
            const uint32_t c = code_at<K>(codes, k);
            const uint32_t kind = c >> 6, lo = c & 7u, ci = (c >> 3) & 7u;
            if (kind == 0u) {
                gax[lo] += gwx;
                gay[lo] += gwy;
            } else if (kind == 1u) {
                gbx[lo] += gwx;
                gby[lo] += gwy;
            } else {
                const int i1 = (ci + 1u < (uint32_t)n1) ? ci + 1 : 0, j1 = (lo + 1u < (uint32_t)n2) ? lo + 1 : 0;
                const R eax = ax[i1] - ax[ci], eay = ay[i1] - ay[ci], ebx = bx[j1] - bx[lo], eby = by[j1] - by[lo];
                const R dx = ax[ci] - bx[lo], dy = ay[ci] - by[lo];
                const R D = eax * eby - eay * ebx, S = ebx * dy - eby * dx, t = S / D;
                const R gt = gwx * eax + gwy * eay;
                const R gS = gt / D, gD = -gt * t / D;
                const R geax = t * gwx + gD * eby, geay = t * gwy - gD * ebx;
                const R gebx = gS * dy - gD * eay, geby = -gS * dx + gD * eax;
                const R gdx = -gS * eby, gdy = gS * ebx;
                gax[ci] += gwx + gdx - geax;
                gay[ci] += gwy + gdy - geay;
                gax[i1] += geax;
                gay[i1] += geay;
                gbx[lo] += -gdx - gebx;
                gby[lo] += -gdy - geby;
                gbx[j1] += gebx;
                gby[j1] += geby;
            }
        }
        for (int v = 0; v < n1; ++v) {
            const int vp = (v == 0) ? n1 - 1 : v - 1, vn = (v + 1 < n1) ? v + 1 : 0;
            gax[v] += (R)0.5 * ga12 * (ay[vn] - ay[vp]);
            gay[v] += (R)0.5 * ga12 * (ax[vp] - ax[vn]);
        }
        for (int v = 0; v < n2; ++v) {
            const int vp = (v == 0) ? n2 - 1 : v - 1, vn = (v + 1 < n2) ? v + 1 : 0;
            gbx[v] += (R)0.5 * ga12 * (by[vn] - by[vp]);
            gby[v] += (R)0.5 * ga12 * (bx[vp] - bx[vn]);
        }
    }
    for (int v = 0; v < K; ++v) {
        const bool ok = err == 0u;
        g1[2 * v] = (ok && v < n1) ? (float)gax[v] : 0.f;
        g1[2 * v + 1] = (ok && v < n1) ? (float)gay[v] : 0.f;
        g2[2 * v] = (ok && v < n2) ? (float)gbx[v] : 0.f;
        g2[2 * v + 1] = (ok && v < n2) ? (float)gby[v] : 0.f;
    }
    return err;
}

// dL/dP1, dL/dP2 from the codes in FP32 (gradients are the same in the local
// frame).  Returns device status bits, or kNeed64 when the pair must be redone
// by bwd_shoelace<K, double>.
constexpr uint32_t kNeed64 = 0x80000000u;

template <int K, bool COUNTS>
__device__ __forceinline__ uint32_t bwd_pair(const Geo<K>& g, float grad, uint32_t nx, const Codes<K>& codes,
                                             bool refine, float (&g1x)[K], float (&g1y)[K], float (&g2x)[K],
                                             float (&g2y)[K]) {
    constexpr int C = 2 * K;
#pragma unroll
    for (int v = 0; v < K; ++v) { g1x[v] = 0.f; g1y[v] = 0.f; g2x[v] = 0.f; g2y[v] = 0.f; }
    if (nx < 3u) return 0u;
    if (nx > (uint32_t)C) return kDevBadFlags;
    const int n1 = g.n1, n2 = g.n2;

    // pass 1: rebuild the intersection vertices
    float wx[C], wy[C];
    bool bad = false;
#pragma unroll
    for (int k = 0; k < C; ++k) {
        wx[k] = 0.f;
        wy[k] = 0.f;
        if ((uint32_t)k < nx) {
            const uint32_t c = code_at<K>(codes, (uint32_t)k);
            const uint32_t kind = c >> 6, lo = c & 7u, ci = (c >> 3) & 7u;
            if (kind == 0u) {
                bad |= (c & 0x3Fu) >= (uint32_t)n1;
                wx[k] = sel<K>(g.ax, lo);
                wy[k] = sel<K>(g.ay, lo);
            } else if (kind == 1u) {
                bad |= (c & 0x3Fu) >= (uint32_t)n2;
                wx[k] = sel<K>(g.bx, lo);
                wy[k] = sel<K>(g.by, lo);
            } else {
                bad |= (kind == 3u) || ci >= (uint32_t)n1 || lo >= (uint32_t)n2;
                const float ax = sel<K>(g.ax, ci), ay = sel<K>(g.ay, ci), eax = sel<K>(g.eax, ci), eay = sel<K>(g.eay, ci);
                const float bx = sel<K>(g.bx, lo), by = sel<K>(g.by, lo), ebx = sel<K>(g.ebx, lo), eby = sel<K>(g.eby, lo);
                const float D = eax * eby - eay * ebx;
                const float S = ebx * (ay - by) - eby * (ax - bx);
                bad |= !(D != 0.f);
                const float t = S / D;
                wx[k] = ax + t * eax;
                wy[k] = ay + t * eay;
            }
        }
    }
    if (bad) return kDevBadFlags;
    float twoA = 0.f, lastx = 0.f, lasty = 0.f;
#pragma unroll
    for (int k = 0; k < C; ++k) {
        if ((uint32_t)k < nx) {
            const float nxx = ((uint32_t)(k + 1) < nx) ? wx[(k + 1) % C] : wx[0];
            const float nxy = ((uint32_t)(k + 1) < nx) ? wy[(k + 1) % C] : wy[0];
            twoA += wx[k] * nxy - wy[k] * nxx;
            if ((uint32_t)k == nx - 1u) { lastx = wx[k]; lasty = wy[k]; }
        }
    }
    float a1, a2;
    input_areas<K, COUNTS>(g, a1, a2);
    const float ai = 0.5f * twoA;
    if (refine) {
        const float L = pair_scale<K, COUNTS>(g);
        if (ai < 1e-6f * L * L) return kNeed64;
    }
    const float U = a1 + a2 - ai;
    if (!(U > 0.f)) return 0u;
    const float rU = 1.0f / U;
    const float gai = grad * (a1 + a2) * rU * rU; // d IoU / d A_i
    const float ga12 = -grad * ai * rU * rU;      // d IoU / d A_1 = d IoU / d A_2

    // pass 2: shoelace adjoint, routed by code
#pragma unroll
    for (int k = 0; k < C; ++k) {
        if ((uint32_t)k < nx) {
            const float pxk = (k == 0) ? lastx : wx[(k + C - 1) % C];
            const float pyk = (k == 0) ? lasty : wy[(k + C - 1) % C];
            const float nxk = ((uint32_t)(k + 1) < nx) ? wx[(k + 1) % C] : wx[0];
            const float nyk = ((uint32_t)(k + 1) < nx) ? wy[(k + 1) % C] : wy[0];
            const float gwx = 0.5f * gai * (nyk - pyk);
            const float gwy = 0.5f * gai * (pxk - nxk);
            const uint32_t c = code_at<K>(codes, (uint32_t)k);
            const uint32_t kind = c >> 6, lo = c & 7u, ci = (c >> 3) & 7u;
            if (kind == 0u) {
                add_at<K>(g1x, lo, gwx);
                add_at<K>(g1y, lo, gwy);
            } else if (kind == 1u) {
                add_at<K>(g2x, lo, gwx);
                add_at<K>(g2y, lo, gwy);
            } else {
                const float ax = sel<K>(g.ax, ci), ay = sel<K>(g.ay, ci), eax = sel<K>(g.eax, ci), eay = sel<K>(g.eay, ci);
                const float bx = sel<K>(g.bx, lo), by = sel<K>(g.by, lo), ebx = sel<K>(g.ebx, lo), eby = sel<K>(g.eby, lo);
                const float dx = ax - bx, dy = ay - by;
                const float D = eax * eby - eay * ebx;
                const float S = ebx * dy - eby * dx;
                const float rD = 1.0f / D;
                const float t = S * rD;
                // w = a + t ea,  t = S / D,  S = cross(eb, a - b),  D = cross(ea, eb)
                const float gt = gwx * eax + gwy * eay;
                const float gS = gt * rD, gD = -gt * t * rD;
                float geax = t * gwx + gD * eby, geay = t * gwy - gD * ebx;
                const float gebx = gS * dy - gD * eay, geby = -gS * dx + gD * eax;
                const float gdx = -gS * eby, gdy = gS * ebx;
                // a_i gets gw + gd - gea; a_{i+1} gets gea; b_j gets -gd - geb; b_{j+1} gets geb
                const uint32_t i1 = (ci + 1u < (uint32_t)n1) ? ci + 1u : 0u;
                const uint32_t j1 = (lo + 1u < (uint32_t)n2) ? lo + 1u : 0u;
                add_at<K>(g1x, ci, gwx + gdx - geax);
                add_at<K>(g1y, ci, gwy + gdy - geay);
                add_at<K>(g1x, i1, geax);
                add_at<K>(g1y, i1, geay);
                add_at<K>(g2x, lo, -gdx - gebx);
                add_at<K>(g2y, lo, -gdy - geby);
                add_at<K>(g2x, j1, gebx);
                add_at<K>(g2y, j1, geby);
            }
        }
    }
    // areas of the inputs
#pragma unroll
    for (int v = 0; v < K; ++v) {
        // previous vertex = this vertex minus the previous edge
        const int pv = (v == 0) ? K - 1 : v - 1;
        float ppx1 = g.ax[pv], ppy1 = g.ay[pv], ppx2 = g.bx[pv], ppy2 = g.by[pv];
        if (COUNTS && v == 0) {
            ppx1 = sel<K>(g.ax, (uint32_t)(n1 - 1));
            ppy1 = sel<K>(g.ay, (uint32_t)(n1 - 1));
            ppx2 = sel<K>(g.bx, (uint32_t)(n2 - 1));
            ppy2 = sel<K>(g.by, (uint32_t)(n2 - 1));
        }
        const float nx1 = g.ax[v] + g.eax[v], ny1 = g.ay[v] + g.eay[v];
        const float nx2 = g.bx[v] + g.ebx[v], ny2 = g.by[v] + g.eby[v];
        const bool v1 = !COUNTS || v < n1, v2 = !COUNTS || v < n2;
        g1x[v] = v1 ? g1x[v] + 0.5f * ga12 * (ny1 - ppy1) : 0.f;
        g1y[v] = v1 ? g1y[v] + 0.5f * ga12 * (ppx1 - nx1) : 0.f;
        g2x[v] = v2 ? g2x[v] + 0.5f * ga12 * (ny2 - ppy2) : 0.f;
        g2y[v] = v2 ? g2y[v] + 0.5f * ga12 * (ppx2 - nx2) : 0.f;
    }
    return 0u;
}

} // namespace dgal
