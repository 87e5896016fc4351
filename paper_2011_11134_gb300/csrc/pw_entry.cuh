// One entry of a pairwise IoU matrix: an exact bounding-box rejection, the
// one-thread fast path (dgal_geom.cuh), and the warp-cooperative robust path
// for the entries the fast path hands back.  Shared by the pairwise matrix
// kernels and the rotated-NMS suppression mask, so both see the same FP32 IoU
// for the same pair of polygons.
#pragma once

#include "dgal_geom.cuh"

namespace dgal {

constexpr int kPwThreads = 128;

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
    if (o.nx >= 3u && U < kThinRel * o.L2) return true; // thin pair: FP64 areas on the warp path
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

} // namespace dgal
