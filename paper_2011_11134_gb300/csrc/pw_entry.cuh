// Entries and tiles of a pairwise IoU matrix: an exact bounding-box
// rejection, the one-thread fast path (dgal_geom.cuh), the warp-cooperative
// robust path for the entries the fast path hands back, and the tile that
// queues the entries whose boxes meet so the clip runs densely.  Shared by the
// pairwise matrix kernels and the rotated-NMS suppression mask, so both see
// the same FP32 IoU for the same pair of polygons.
#pragma once

#include "dgal_geom.cuh"

namespace dgal {

constexpr int kPwThreads = 128;
// Most warps a pairwise tile block may have (pw_tile keeps one queue count per warp).
constexpr int kPwMaxWarps = 8;

// Fast path for one matrix entry.  Returns true when the entry must be
// finished by the warp-cooperative robust path; otherwise sets iou / nxo.
// `refine`: FP64 signs for orientations too small for FP32 (fwd_generic).
template <int K, bool COUNTS>
__device__ __forceinline__ bool pw_fast(const float* __restrict__ pa, const float* __restrict__ pb, int n1, int n2,
                                        float& iou, uint32_t& nxo, uint32_t& err, bool refine) {
    iou = 0.f;
    nxo = 0u;
    if (COUNTS && (n1 < 3 || n1 > K || n2 < 3 || n2 > K)) {
        err |= kDevBadCount;
        return false;
    }
    float px[K], py[K], qx[K], qy[K];
    load_poly<K>(pa, px, py);
    load_poly<K>(pb, qx, qy);
    float ax0 = px[0], ax1 = px[0], ay0 = py[0], ay1 = py[0];
    float bx0 = qx[0], bx1 = qx[0], by0 = qy[0], by1 = qy[0];
#pragma unroll
    for (int v = 1; v < K; ++v) {
        const bool va = !COUNTS || v < n1, vb = !COUNTS || v < n2;
        ax0 = va ? fminf(ax0, px[v]) : ax0;
        ax1 = va ? fmaxf(ax1, px[v]) : ax1;
        ay0 = va ? fminf(ay0, py[v]) : ay0;
        ay1 = va ? fmaxf(ay1, py[v]) : ay1;
        bx0 = vb ? fminf(bx0, qx[v]) : bx0;
        bx1 = vb ? fmaxf(bx1, qx[v]) : bx1;
        by0 = vb ? fminf(by0, qy[v]) : by0;
        by1 = vb ? fmaxf(by1, qy[v]) : by1;
    }
    if (ax1 < bx0 || bx1 < ax0 || ay1 < by0 || by1 < ay0) return false;
    Geo<K> g;
    FwdOut<K> o;
    make_geo<K, COUNTS>(px, py, qx, qy, n1, n2, g);
    input_areas<K, COUNTS>(g, o.a1, o.a2);
    if (!(refine ? fwd_generic<K, COUNTS>(g, o, pa, pb) : fwd_generic<K, COUNTS>(g, o))) return true;
    const float U = o.a1 + o.a2 - o.ai;
    if (o.nx >= 3u && U < kThinRel * o.L2) return true; // thin pair: float-float areas on the warp path
    nxo = o.nx;
    iou = (o.nx >= 3u && U > 0.f) ? o.ai / U : 0.f;
    return false;
}

// Finishes the entries of this warp step that the fast path handed back, one
// at a time with the whole warp; the owning lane stores the result.
template <int K>
__device__ __forceinline__ void pw_finish(unsigned todo, const float* __restrict__ pa, const float* __restrict__ pb,
                                          int n1, int n2, bool refine, float& iou, uint32_t& nxo, uint32_t& err) {
    const int lane = threadIdx.x & 31;
    while (todo) {
        const int src = __ffs(todo) - 1;
        todo &= todo - 1;
        const float* qa = (const float*)__shfl_sync(0xffffffffu, (unsigned long long)pa, src);
        const float* qb = (const float*)__shfl_sync(0xffffffffu, (unsigned long long)pb, src);
        const int m1 = __shfl_sync(0xffffffffu, n1, src), m2 = __shfl_sync(0xffffffffu, n2, src);
        FwdOut<K> o;
        o.err = 0;
        warp_robust<K>(qa, qb, m1, m2, refine, o);
        if (lane == src) {
            err |= o.err;
            iou = o.iou;
            nxo = o.nx;
        }
    }
}

// Axis-aligned bounding box (min x, min y, max x, max y) of a polygon's first
// n vertices; a count outside [3, K] gives a box that meets every box, so the
// entry reaches pw_fast, which reports the count.
template <int K, bool COUNTS> __device__ __forceinline__ float4 poly_box(const float* __restrict__ p, int n) {
    if (COUNTS && (n < 3 || n > K)) {
        const float inf = __int_as_float(0x7f800000);
        return make_float4(-inf, -inf, inf, inf);
    }
    float x[K], y[K];
    load_poly<K>(p, x, y);
    float4 r = make_float4(x[0], y[0], x[0], y[0]);
#pragma unroll
    for (int v = 1; v < K; ++v) {
        const bool on = !COUNTS || v < n;
        r.x = on ? fminf(r.x, x[v]) : r.x;
        r.y = on ? fminf(r.y, y[v]) : r.y;
        r.z = on ? fmaxf(r.z, x[v]) : r.z;
        r.w = on ? fmaxf(r.w, y[v]) : r.w;
    }
    return r;
}

// Where a tile's results go: the IoU matrix (and nx) of one N x M matrix.
// wanted(i, j): the entry is computed at all; disjoint(i, j): its boxes do
// not meet (IoU 0, nx 0 by definition); put(i, j, iou, nx): the clip's result.
struct PwMatrixOut {
    float* __restrict__ iou;
    uint8_t* __restrict__ nx; // nullable
    int64_t M;
    __device__ __forceinline__ bool wanted(int64_t, int64_t) const { return true; }
    __device__ __forceinline__ void disjoint(int64_t i, int64_t j) const {
        iou[i * M + j] = 0.f;
        if (nx) nx[i * M + j] = 0;
    }
    __device__ __forceinline__ void put(int64_t i, int64_t j, float v, uint32_t c) const {
        iou[i * M + j] = v;
        if (nx) nx[i * M + j] = (uint8_t)c;
    }
};

// One tile of rows [i0, i0 + R) x columns [j0, j0 + blockDim.x) of an N x M
// matrix (a, b: the matrix's row and column polygons; out: where results go):
//   1. thread c computes the bounding box of column j0 + c, threads < R those
//      of the tile's rows (shared memory);
//   2. every wanted entry is tested on the boxes (exact comparisons of the
//      float inputs); a disjoint pair has IoU 0 and nx 0 by definition and is
//      reported at once (consecutive threads, consecutive columns), the others
//      are queued in shared memory (codes r << 8 | c).  Each warp queues its
//      own 32 columns in its own region of s_q (R x 32 codes at w R 32) with a
//      running count in a register (a ballot and a prefix count per row, no
//      shared-memory atomic), and leaves its count in s_nq[w];
//   3. the block's warps clip the queued entries densely (pw_fast, with the
//      warp-cooperative finish for the ones it hands back), reading the warps'
//      regions as one queue.
// In bird's-eye scenes about 2% of the entries have meeting boxes; without the
// queue a warp runs the clip whenever one of its 32 entries needs it.  Every
// thread of the block calls this (it has block barriers); blockDim.x is a
// multiple of 32 and at most kPwMaxWarps * 32, R <= 256 (8-bit fields of the
// queue codes); s_q holds R x blockDim.x codes, s_nq one count per warp.
template <int K, bool COUNTS, class Out>
__device__ __forceinline__ void pw_tile(const float* __restrict__ a, const uint8_t* __restrict__ ca, int64_t N,
                                        const float* __restrict__ b, const uint8_t* __restrict__ cb, int64_t M,
                                        int64_t i0, int64_t j0, int R, float4* s_rbox, uint16_t* s_q, int* s_nq,
                                        bool refine, uint32_t& err, const Out& out) {
    constexpr unsigned full = 0xffffffffu;
    const int t = threadIdx.x, lane = t & 31, C = blockDim.x;
    const float inf = __int_as_float(0x7f800000);
    const int64_t j = j0 + t;
    const bool jv = j < M;
    const float4 cbx = jv ? poly_box<K, COUNTS>(b + j * 2 * K, (COUNTS && cb) ? (int)cb[j] : K)
                          : make_float4(inf, inf, -inf, -inf);
    if (t < R) {
        const int64_t i = i0 + t;
        s_rbox[t] = (i < N) ? poly_box<K, COUNTS>(a + i * 2 * K, (COUNTS && ca) ? (int)ca[i] : K)
                            : make_float4(inf, inf, -inf, -inf);
    }
    __syncthreads();
    const int w = t >> 5, nw = C >> 5;
    uint16_t* q_w = s_q + w * R * 32;
    const unsigned below = (1u << lane) - 1u;
    int cnt = 0;
#pragma unroll 4
    for (int r = 0; r < R; ++r) {
        const int64_t i = i0 + r;
        const bool v = jv && i < N && out.wanted(i, j);
        const float4 rbx = s_rbox[r];
        const bool meet = v && !(rbx.z < cbx.x || cbx.z < rbx.x || rbx.w < cbx.y || cbx.w < rbx.y);
        if (v && !meet) out.disjoint(i, j);
        const unsigned bal = __ballot_sync(full, meet);
        if (meet) q_w[cnt + __popc(bal & below)] = (uint16_t)((r << 8) | t);
        cnt += __popc(bal);
    }
    if (lane == 0) s_nq[w] = cnt;
    __syncthreads();
    int nq = 0;
    for (int u = 0; u < nw; ++u) nq += s_nq[u];
    for (int qb = t & ~31; qb < nq; qb += C) {
        const int q = qb + lane;
        const bool act = q < nq;
        // entry q of the joined queue: warp src's entry rem (the counts are
        // read from shared memory, so they take no registers)
        int src = 0, rem = q;
        for (int u = 0; u + 1 < nw; ++u) {
            const int c = s_nq[u];
            const bool past = src == u && rem >= c;
            rem -= past ? c : 0;
            src += past ? 1 : 0;
        }
        const int code = act ? (int)s_q[src * R * 32 + rem] : 0;
        const int64_t i = i0 + (code >> 8), jj = j0 + (code & 0xFF);
        const int n1 = (COUNTS && ca && act) ? (int)ca[i] : K;
        const int n2 = (COUNTS && cb && act) ? (int)cb[jj] : K;
        const float* pa = a + (act ? i : 0) * 2 * K;
        const float* pb = b + (act ? jj : 0) * 2 * K;
        float v = 0.f;
        uint32_t c = 0;
        const bool hard = act && pw_fast<K, COUNTS>(pa, pb, n1, n2, v, c, err, refine);
        pw_finish<K>(__ballot_sync(full, hard), pa, pb, n1, n2, refine, v, c, err);
        if (act) out.put(i, jj, v, c);
    }
    __syncthreads(); // the next tile reuses the boxes and the queue
}

} // namespace dgal
