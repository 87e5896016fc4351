// Paired IoU kernels and their launch templates (included by paired.cu for
// the 2D IoU and by paired3d.cu for the 3D IoU, so each translation unit
// instantiates its own half).
//
// Forward (paper Sec. II-B `iou`): loads both polygons with 128-bit loads,
// clips in registers (dgal_geom.cuh), stores IoU (4 B), nx (1 B) and the
// 2K code bytes as one 64/128-bit store, plus an optional degeneracy byte.
// Backward (paper Sec. II-B `iou_backward`): reads the polygons, dL/dIoU and
// the recorded (nx, xflags), or recomputes the clip, and writes both
// gradients with 128-bit stores.  One-pass form (k_paired_fused, K = 4): both
// halves in one kernel for pairs in pinned host memory, the codes kept in
// registers between them.
#pragma once

#include "dgal_geom.cuh"
#include "dgal_internal.h"
#include "group8.cuh"

#include <type_traits>

namespace dgal {

constexpr int kPairThreads = 128;

template <int K> __device__ __forceinline__ void store_codes(uint8_t* __restrict__ xf, int64_t k, const Codes<K>& c) {
    if constexpr (K == 4) {
        reinterpret_cast<uint64_t*>(xf)[k] = c.w[0];
    } else {
        reinterpret_cast<uint4*>(xf)[k] =
            make_uint4((uint32_t)c.w[0], (uint32_t)(c.w[0] >> 32), (uint32_t)c.w[1], (uint32_t)(c.w[1] >> 32));
    }
}

template <int K> __device__ __forceinline__ void load_codes(const uint8_t* __restrict__ xf, int64_t k, Codes<K>& c) {
    if constexpr (K == 4) {
        c.w[0] = __ldg(reinterpret_cast<const unsigned long long*>(xf) + k);
    } else {
        uint4 u = __ldg(reinterpret_cast<const uint4*>(xf) + k);
        c.w[0] = (uint64_t)u.x | ((uint64_t)u.y << 32);
        c.w[1] = (uint64_t)u.z | ((uint64_t)u.w << 32);
    }
}

template <int K> __device__ __forceinline__ void store_poly(float* __restrict__ p, const float (&x)[K], const float (&y)[K]) {
    float4* q = reinterpret_cast<float4*>(p);
#pragma unroll
    for (int v = 0; v < K / 2; ++v) q[v] = make_float4(x[2 * v], y[2 * v], x[2 * v + 1], y[2 * v + 1]);
}

// The K = 4 kernels walk the pairs warp by warp (32 consecutive pairs per
// warp and step, grid-stride over warps), with no block-wide barrier.  In the
// forward, a pair the fast path cannot finish (a sign pattern two convex
// polygons in general position cannot have, a thin pair, or without
// refinement a near-degenerate one; well under 0.1% of random boxes) is finished right after the
// step by the whole warp (warp_robust, a non-inlined call, so its registers
// and slow-path code stay off the common path); the SM keeps issuing from its
// other warps meanwhile.  In the backward, a pair whose codes the shape
// derivative cannot take (not in general position, or with refinement a tiny
// intersection) takes the shoelace adjoint after the rest, with the whole
// warp on it (warp_bwd).  The K = 8 group forward instead marks such pairs
// and leaves them to a launch of their own (k_paired_fwd_finish).

// IoU-loss mode of the paired kernels (paper Sec. IV-A, the IoU loss over
// rotated boxes): the forward adds scale * w_k (1 - IoU_k) into one partial
// per warp, and the backward takes dL/dIoU_k = -scale * w_k * dloss (w = 1
// when weight is NULL, dloss = 1 when NULL) instead of reading an upstream
// gradient.  For the GIoU loss the forward also keeps each pair's union U and
// the backward adds scale * w_k * dloss / A_h to dL/dA_i and subtracts it from
// dL/dA_1, dL/dA_2 (A_h the pair's hull area, from the GIoU pass).
struct LossArgs {
    const float* weight;
    float scale;
    float* partials;        // one float per warp of the forward grid
    float* loss;            // backward: block 0 writes the sum of the partials here (NULL: not in this launch)
    int64_t nparts;         // number of partials
    float* u_out;           // forward, GIoU: U = A_1 + A_2 - A_i per pair (NULL: not kept)
    const float* ah;        // backward, GIoU: hull area per pair (NULL: plain IoU loss)
    const float* partials2; // backward: partials of the GIoU / DIoU terms, folded after the first (or NULL)
    int64_t nparts2;
    const float* dloss;     // backward: device pointer to the upstream gradient of the loss (NULL: 1)
};

// dL/dIoU_k of the loss-mode backward.
__device__ __forceinline__ float loss_dl(const LossArgs& la, float w) {
    return -la.scale * w * (la.dloss ? __ldg(la.dloss) : 1.f);
}

// 3D mode of the paired kernels: each box also has a vertical extent
// (z_center, height) in z1 / z2 (float [n][2]); the forward gives the 3D IoU
// and the backward also writes dL/d(z_center, height) into gz1 / gz2.
struct ZArgs {
    const float* z1;
    const float* z2;
    float* gz1;
    float* gz2;
};

__device__ __forceinline__ ZPair z_of(const ZArgs& za, int64_t k) {
    return z_pair(__ldg(reinterpret_cast<const float2*>(za.z1) + k), __ldg(reinterpret_cast<const float2*>(za.z2) + k));
}

template <bool Z3> struct AdjOf { typedef AdjIou T; };
template <> struct AdjOf<true> { typedef AdjIou3 T; };

// The adjoint policy of pair k for dL/dIoU = g.
template <bool Z3> __device__ __forceinline__ typename AdjOf<Z3>::T adj_of(float g, const ZArgs& za, int64_t k) {
    typename AdjOf<Z3>::T a;
    a.g = g;
    if constexpr (Z3) {
        a.z = z_of(za, k);
        a.hit = false;
        a.ai = a.a1 = a.a2 = 0.f;
    } else {
        a.e = 0.f;
    }
    return a;
}

// Writes dL/d(z_center, height) of pair k (3D mode only).
template <bool Z3> __device__ __forceinline__ void put_zgrad(const ZArgs& za, int64_t k, const typename AdjOf<Z3>::T& a) {
    if constexpr (Z3) {
        float2 u, v;
        a.z_grads(u, v);
        reinterpret_cast<float2*>(za.gz1)[k] = u;
        reinterpret_cast<float2*>(za.gz2)[k] = v;
    }
}

__device__ __forceinline__ float loss_weight(const LossArgs& la, int64_t k) {
    return la.weight ? __ldg(la.weight + k) : 1.f;
}

// The adjoint policy of pair k in a backward: dL/dIoU read from grad, or in
// loss mode formed from the weights (plus the GIoU term when la.ah is set).
template <bool LOSS, bool Z3>
__device__ __forceinline__ typename AdjOf<Z3>::T make_adj(const LossArgs& la, const float* __restrict__ grad,
                                                          const ZArgs& za, int64_t k) {
    if constexpr (LOSS) {
        const float g = loss_dl(la, loss_weight(la, k));
        auto a = adj_of<Z3>(g, za, k);
        if constexpr (!Z3) {
            if (la.ah) a.e = -g / __ldg(la.ah + k);
        }
        return a;
    } else {
        return adj_of<Z3>(__ldg(grad + k), za, k);
    }
}

__device__ __forceinline__ void put_partial(const LossArgs& la, float acc) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) la.partials[((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5] = acc;
}

// Block 0 of the loss-mode backward sums the forward's per-warp partials in a
// fixed order before taking its pairs: thread t adds float4 blocks t,
// t + blockDim, ... (four loads in flight per round, each block's values in
// order), then the scalar tail, then a fixed tree over the warps.  The order
// does not depend on scheduling, so the loss is deterministic, and the sum
// needs no launch of its own: the other blocks go straight to their pairs.
// partials must be 16-byte aligned.  Block-uniform (it has block barriers).
// Thread-level part of the fixed-order sum of m partials (16-byte aligned).
__device__ __forceinline__ float fold_part(const float* __restrict__ partials, int64_t m) {
    const int64_t m4 = m / 4, step = blockDim.x;
    const float4* p4 = reinterpret_cast<const float4*>(partials);
    float v = 0.f;
    for (int64_t base = 0; base < m4; base += 4 * step) {
        float4 a[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t i = base + u * step + threadIdx.x;
            a[u] = (i < m4) ? __ldg(p4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) v += (a[u].x + a[u].y) + (a[u].z + a[u].w);
    }
    for (int64_t i = 4 * m4 + threadIdx.x; i < m; i += step) v += partials[i];
    return v;
}

__device__ __forceinline__ void loss_fold(const LossArgs& la) {
    if (!la.loss || blockIdx.x != 0) return;
    __shared__ float sh[32];
    float v = fold_part(la.partials, la.nparts);
    if (la.partials2) v += fold_part(la.partials2, la.nparts2);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
        if (l == 0) *la.loss = t;
    }
}

// Stores the forward results of pair k (and adds its loss term in loss mode).
template <int K, bool SAVE, bool LOSS>
__device__ __forceinline__ void put_fwd(const FwdOut<K>& o, int64_t k, float w, const LossArgs& la,
                                        float* __restrict__ iou, uint8_t* __restrict__ nx,
                                        uint8_t* __restrict__ xflags, uint8_t* __restrict__ degen, float& acc) {
    if (LOSS) {
        acc += la.scale * w * (1.f - o.iou);
        if (la.u_out) la.u_out[k] = o.a1 + o.a2 - (o.nx >= 3u ? o.ai : 0.f);
    }
    if (!LOSS || iou) iou[k] = o.iou;
    if (SAVE) {
        nx[k] = (uint8_t)o.nx;
        store_codes<K>(xflags, k, o.codes);
    }
    if (degen) degen[k] = (uint8_t)o.degen;
}

// Minimum resident blocks per SM of the paired kernels (a register cap),
// each measured on its workload's step.  K = 4: the forward at 7 blocks (72
// registers) and the backward at 6 (80 registers) were fastest; the
// backward lost 2 and 4 us at 7 and 8 blocks, and 5 blocks were slower for
// both.  The backward that recomputes the clip carries the forward's code as
// well and keeps 4 blocks (128 registers).
constexpr int kFwdMinBlocks = 7;
constexpr int kBwdMinBlocks = 6;
// the K = 8 group forward: 8 blocks of 128 per SM (64 registers), measured
// faster than 5 to 7
constexpr int kFwdG8MinBlocks = 8;
// the K = 8 group backward: 10 blocks of 128 per SM (48 registers) measured
// faster than 5 to 8 or 12, despite the register spills it brings
constexpr int kBwdG8MinBlocks = 10;

template <int K, bool COUNTS, bool SAVE, bool LOSS, bool Z3>
__global__ void __launch_bounds__(kPairThreads, kFwdMinBlocks)
k_paired_fwd(const float* __restrict__ p1, const uint8_t* __restrict__ c1, const float* __restrict__ p2,
             const uint8_t* __restrict__ c2, int64_t n, float* __restrict__ iou, uint8_t* __restrict__ nx,
             uint8_t* __restrict__ xflags, uint8_t* __restrict__ degen, uint32_t flags, uint32_t* status,
             LossArgs la, ZArgs za) {
    constexpr unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * kPairThreads;
    const bool refine = (flags & kFlagRefine) && !(flags & kFlagPlain);
    // a backward launched right after this grid with programmatic stream
    // serialisation may be scheduled once every block of this grid has started
    // (it waits for this grid's completion before touching memory)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    uint32_t err = 0;
    float acc = 0.f;
    for (int64_t base = (int64_t)blockIdx.x * kPairThreads + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t k = base + lane;
        int n1 = K, n2 = K;
        bool hard = false;
        float w = 0.f;
        if (k < n) {
            if (LOSS) w = loss_weight(la, k);
            if (COUNTS) {
                n1 = c1 ? (int)c1[k] : K;
                n2 = c2 ? (int)c2[k] : K;
            }
            FwdOut<K> o;
            if (COUNTS && (n1 < 3 || n1 > K || n2 < 3 || n2 > K)) {
                err |= kDevBadCount;
                o.nx = 0;
                o.iou = 0.f;
                o.ai = o.a1 = o.a2 = 0.f;
                o.degen = 0;
                codes_fill<K>(o.codes, ~0ull);
            } else {
                float px[K], py[K], qx[K], qy[K];
                load_poly<K>(p1 + k * 2 * K, px, py);
                load_poly<K>(p2 + k * 2 * K, qx, qy);
                Geo<K> g;
                make_geo<K, COUNTS>(px, py, qx, qy, n1, n2, g);
                input_areas<K, COUNTS>(g, o.a1, o.a2);
                o.degen = 0;
                hard = refine ? !fwd_generic<K, COUNTS>(g, o, p1 + k * 2 * K, p2 + k * 2 * K)
                              : !fwd_generic<K, COUNTS>(g, o);
                // thin pairs: float-float areas on the warp path (kThinRel)
                hard = hard || (o.nx >= 3u && o.a1 + o.a2 - o.ai < kThinRel * o.L2);
                if (!hard) {
                    if constexpr (Z3) {
                        o.iou = iou3_value(o.ai, o.a1, o.a2, o.nx, z_of(za, k));
                    } else {
                        const float U = o.a1 + o.a2 - o.ai;
                        o.iou = (o.nx >= 3u && U > 0.f) ? o.ai / U : 0.f;
                    }
                }
            }
            if (!hard) put_fwd<K, SAVE, LOSS>(o, k, w, la, iou, nx, xflags, degen, acc);
        }
        // pairs the fast path hands back (near-degenerate or not in general
        // position): finished here, one at a time, by the whole warp
        unsigned todo = __ballot_sync(full, hard);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t kk = base + src;
            const int m1 = __shfl_sync(full, n1, src), m2 = __shfl_sync(full, n2, src);
            FwdOut<K> o;
            o.err = 0;
            warp_robust<K>(p1 + kk * 2 * K, p2 + kk * 2 * K, m1, m2, refine, o);
            if (lane == src) {
                if constexpr (Z3) o.iou = iou3_value(o.ai, o.a1, o.a2, o.nx, z_of(za, kk));
                err |= o.err;
                put_fwd<K, SAVE, LOSS>(o, kk, w, la, iou, nx, xflags, degen, acc);
            }
        }
    }
    if (LOSS) put_partial(la, acc);
    if (err) atomicOr(status, err);
}

template <int K, bool COUNTS, bool RECOMPUTE, bool LOSS, bool Z3>
__global__ void __launch_bounds__(kPairThreads, RECOMPUTE ? 4 : kBwdMinBlocks)
k_paired_bwd(const float* __restrict__ p1, const uint8_t* __restrict__ c1, const float* __restrict__ p2,
             const uint8_t* __restrict__ c2, int64_t n, const float* __restrict__ grad,
             const uint8_t* __restrict__ nxs, const uint8_t* __restrict__ xflags, float* __restrict__ g1,
             float* __restrict__ g2, uint32_t flags, uint32_t* status, LossArgs la, ZArgs za) {
    constexpr unsigned full = 0xffffffffu;
    __shared__ float s_bwd[kPairThreads / 32][4 * K];
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * kPairThreads;
    const bool refine = (flags & kFlagRefine) && !(flags & kFlagPlain);
    // Launched with programmatic stream serialisation (launch_pdl), the blocks
    // may start while the grid before this one (the forward) is finishing:
    // wait for its completion and its memory before the first global access,
    // so no input, including the flags and partials it wrote, is read early.
    // Without that launch attribute this returns at once.
    asm volatile("griddepcontrol.wait;" ::: "memory");
    if constexpr (LOSS) loss_fold(la);
    uint32_t err = 0;
    for (int64_t base = (int64_t)blockIdx.x * kPairThreads + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t k = base + lane;
        int n1 = K, n2 = K;
        bool slow = false, needfwd = false;
        Codes<K> codes;
        uint32_t nxk = 0;
        if (k < n) {
            if (COUNTS) {
                n1 = c1 ? (int)c1[k] : K;
                n2 = c2 ? (int)c2[k] : K;
            }
            float g1x[K], g1y[K], g2x[K], g2y[K];
            auto adj = make_adj<LOSS, Z3>(la, grad, za, k);
            if (COUNTS && (n1 < 3 || n1 > K || n2 < 3 || n2 > K)) {
                err |= kDevBadCount;
#pragma unroll
                for (int v = 0; v < K; ++v) { g1x[v] = g1y[v] = g2x[v] = g2y[v] = 0.f; }
            } else {
                float px[K], py[K], qx[K], qy[K];
                load_poly<K>(p1 + k * 2 * K, px, py);
                load_poly<K>(p2 + k * 2 * K, qx, qy);
                Geo<K> g;
                make_geo<K, COUNTS>(px, py, qx, qy, n1, n2, g);
                bool have = true;
                if (RECOMPUTE) {
                    FwdOut<K> o;
                    have = refine ? fwd_generic<K, COUNTS>(g, o, p1 + k * 2 * K, p2 + k * 2 * K)
                                  : fwd_generic<K, COUNTS>(g, o);
                    codes = o.codes;
                    nxk = o.nx;
                } else {
                    nxk = nxs[k];
                    load_codes<K>(xflags, k, codes);
                }
                uint32_t e = kSlow;
                if (have) e = bwd_shape<K, COUNTS>(g, adj, nxk, codes, refine, g1x, g1y, g2x, g2y);
                needfwd = !have;
                slow = (e == kSlow);
                if (!slow) err |= e;
            }
            if (!slow) {
                store_poly<K>(g1 + k * 2 * K, g1x, g1y);
                store_poly<K>(g2 + k * 2 * K, g2x, g2y);
                put_zgrad<Z3>(za, k, adj);
            }
        }
        if (RECOMPUTE) {
            unsigned todo = __ballot_sync(full, needfwd);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const int64_t kk = base + src;
                const int m1 = __shfl_sync(full, n1, src), m2 = __shfl_sync(full, n2, src);
                FwdOut<K> o;
                o.err = 0;
                warp_robust<K>(p1 + kk * 2 * K, p2 + kk * 2 * K, m1, m2, refine, o);
                if (lane == src) {
                    err |= o.err;
                    codes = o.codes;
                    nxk = o.nx;
                }
            }
        }
        unsigned todo = __ballot_sync(full, slow);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t kk = base + src;
            const int m1 = __shfl_sync(full, n1, src), m2 = __shfl_sync(full, n2, src);
            const uint32_t mnx = __shfl_sync(full, nxk, src);
            Codes<K> cs;
#pragma unroll
            for (int q = 0; q < (2 * K + 7) / 8; ++q) cs.w[q] = __shfl_sync(full, codes.w[q], src);
            auto a = make_adj<LOSS, Z3>(la, grad, za, kk);
            const uint32_t e = refine ? warp_bwd<K, ff>(p1 + kk * 2 * K, p2 + kk * 2 * K, m1, m2, a, mnx, cs,
                                                            g1 + kk * 2 * K, g2 + kk * 2 * K, s_bwd[threadIdx.x >> 5])
                                      : warp_bwd<K, float>(p1 + kk * 2 * K, p2 + kk * 2 * K, m1, m2, a, mnx, cs,
                                                           g1 + kk * 2 * K, g2 + kk * 2 * K, s_bwd[threadIdx.x >> 5]);
            if (lane == src) {
                err |= e;
                put_zgrad<Z3>(za, kk, a);
            }
        }
    }
    if (err) atomicOr(status, err);
}

// Forward and backward in one pass, for pairs that live in pinned host
// memory the kernel reads and writes in place: the step is then bound by the
// host link, and the clip state stays in registers between the two halves
// instead of making a round trip as flags.  Every value is the one the
// separate kernels give: the forward is k_paired_fwd's (with its hand-back of
// hard pairs to warp_robust), and the backward is k_paired_bwd's from the
// codes the forward just produced.
template <int K, bool COUNTS>
__global__ void __launch_bounds__(kPairThreads, 4)
k_paired_fused(const float* __restrict__ p1, const uint8_t* __restrict__ c1, const float* __restrict__ p2,
               const uint8_t* __restrict__ c2, int64_t n, const float* __restrict__ grad, float* __restrict__ iou,
               float* __restrict__ g1, float* __restrict__ g2, uint32_t flags, uint32_t* status) {
    constexpr unsigned full = 0xffffffffu;
    __shared__ float s_bwd[kPairThreads / 32][4 * K];
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * kPairThreads;
    const bool refine = (flags & kFlagRefine) && !(flags & kFlagPlain);
    const ZArgs za{nullptr, nullptr, nullptr, nullptr};
    uint32_t err = 0;
    for (int64_t base = (int64_t)blockIdx.x * kPairThreads + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t k = base + lane;
        const bool live = k < n;
        int n1 = K, n2 = K;
        if (COUNTS && live) {
            n1 = c1 ? (int)c1[k] : K;
            n2 = c2 ? (int)c2[k] : K;
        }
        const bool good = live && (!COUNTS || (n1 >= 3 && n1 <= K && n2 >= 3 && n2 <= K));
        float px[K], py[K], qx[K], qy[K];
        FwdOut<K> o;
        o.iou = 0.f;
        bool hard = false;
        if (good) {
            load_poly<K>(p1 + k * 2 * K, px, py);
            load_poly<K>(p2 + k * 2 * K, qx, qy);
            Geo<K> g;
            make_geo<K, COUNTS>(px, py, qx, qy, n1, n2, g);
            input_areas<K, COUNTS>(g, o.a1, o.a2);
            hard = refine ? !fwd_generic<K, COUNTS>(g, o, p1 + k * 2 * K, p2 + k * 2 * K)
                          : !fwd_generic<K, COUNTS>(g, o);
            hard = hard || (o.nx >= 3u && o.a1 + o.a2 - o.ai < kThinRel * o.L2);
            if (!hard) {
                const float U = o.a1 + o.a2 - o.ai;
                o.iou = (o.nx >= 3u && U > 0.f) ? o.ai / U : 0.f;
            }
        } else if (live) {
            err |= kDevBadCount;
        }
        unsigned todo = __ballot_sync(full, hard);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t kk = base + src;
            const int m1 = __shfl_sync(full, n1, src), m2 = __shfl_sync(full, n2, src);
            FwdOut<K> r;
            r.err = 0;
            warp_robust<K>(p1 + kk * 2 * K, p2 + kk * 2 * K, m1, m2, refine, r);
            if (lane == src) {
                err |= r.err;
                o.iou = r.iou;
                o.nx = r.nx;
                o.codes = r.codes;
            }
        }
        bool slow = false;
        if (live) {
            iou[k] = o.iou;
            float g1x[K], g1y[K], g2x[K], g2y[K];
            if (good) {
                Geo<K> g;
                make_geo<K, COUNTS>(px, py, qx, qy, n1, n2, g);
                auto adj = adj_of<false>(grad[k], za, k);
                const uint32_t e = bwd_shape<K, COUNTS>(g, adj, o.nx, o.codes, refine, g1x, g1y, g2x, g2y);
                slow = e == kSlow;
                if (!slow) err |= e;
            } else {
#pragma unroll
                for (int v = 0; v < K; ++v) { g1x[v] = g1y[v] = g2x[v] = g2y[v] = 0.f; }
            }
            if (!slow) {
                store_poly<K>(g1 + k * 2 * K, g1x, g1y);
                store_poly<K>(g2 + k * 2 * K, g2x, g2y);
            }
        }
        todo = __ballot_sync(full, slow);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t kk = base + src;
            const int m1 = __shfl_sync(full, n1, src), m2 = __shfl_sync(full, n2, src);
            const uint32_t mnx = __shfl_sync(full, o.nx, src);
            Codes<K> cs;
#pragma unroll
            for (int q = 0; q < (2 * K + 7) / 8; ++q) cs.w[q] = __shfl_sync(full, o.codes.w[q], src);
            auto a = adj_of<false>(grad[kk], za, kk);
            const uint32_t e = refine ? warp_bwd<K, ff>(p1 + kk * 2 * K, p2 + kk * 2 * K, m1, m2, a, mnx, cs,
                                                            g1 + kk * 2 * K, g2 + kk * 2 * K, s_bwd[threadIdx.x >> 5])
                                      : warp_bwd<K, float>(p1 + kk * 2 * K, p2 + kk * 2 * K, m1, m2, a, mnx, cs,
                                                           g1 + kk * 2 * K, g2 + kk * 2 * K, s_bwd[threadIdx.x >> 5]);
            if (lane == src) err |= e;
        }
    }
    if (err) atomicOr(status, err);
}

// K = 8: one group of 8 lanes per pair (group8.cuh), 4 pairs per warp and
// step, grid-stride over warps.  Pairs the group cannot finish are done by the
// whole warp (forward) or by the group's first lane (backward) afterwards.
// DEFER: a pair the group hands back is marked (its IoU written as NaN) and
// left to k_paired_fwd_finish, instead of being finished here by the warp.
// KIN: the capacity of the stored polygons (8; or 4, quadrilaterals spread
// over 8 lanes to cut the latency of small batches).
template <bool SAVE, bool LOSS, bool Z3, bool DEFER = false, int KIN = 8>
__global__ void __launch_bounds__(kPairThreads, kFwdG8MinBlocks)
k_paired_fwd_g8(const float* __restrict__ p1, const uint8_t* __restrict__ c1, const float* __restrict__ p2,
                const uint8_t* __restrict__ c2, int64_t n, float* __restrict__ iou, uint8_t* __restrict__ nx,
                uint8_t* __restrict__ xflags, uint8_t* __restrict__ degen, uint32_t flags, uint32_t* status,
                LossArgs la, ZArgs za) {
    const int lane = threadIdx.x & 31, r = lane & 7;
    const bool refine = (flags & kFlagRefine) && !(flags & kFlagPlain);
    const int64_t warp = ((int64_t)blockIdx.x * kPairThreads + threadIdx.x) >> 5;
    const int64_t stride = (int64_t)gridDim.x * (kPairThreads / 32) * 4;
    uint32_t err = 0;
    float acc = 0.f;
    for (int64_t base = warp * 4; base < n; base += stride) {
        const int64_t k = base + (lane >> 3);
        const bool act = k < n;
        const int n1 = (act && c1) ? (int)c1[k] : KIN, n2 = (act && c2) ? (int)c2[k] : KIN;
        const bool good = act && n1 >= 3 && n1 <= KIN && n2 >= 3 && n2 <= KIN;
        bool hard = false;
        const float w = (LOSS && act && r == 0) ? loss_weight(la, k) : 0.f;
        if (good) {
            g8::Lane L;
            g8::load_lane<KIN>(p1 + k * 2 * KIN, p2 + k * 2 * KIN, n1, n2, r, L);
            g8::FwdG o;
            hard = refine ? !g8::fwd_group<KIN>(L, o, p1 + k * 2 * KIN, p2 + k * 2 * KIN) : !g8::fwd_group<KIN>(L, o);
            if constexpr (Z3) {
                if (!hard && r == 0) o.iou = iou3_value(o.ai, o.a1, o.a2, o.nx, z_of(za, k));
            }
            if (!hard && r == 0) {
                if (LOSS) {
                    acc += la.scale * w * (1.f - o.iou);
                    if (la.u_out) la.u_out[k] = o.a1 + o.a2 - (o.nx >= 3u ? o.ai : 0.f);
                }
                if (!LOSS || iou) iou[k] = o.iou;
                if (SAVE) {
                    nx[k] = (uint8_t)o.nx;
                    if constexpr (KIN == 8)
                        reinterpret_cast<uint4*>(xflags)[k] =
                            make_uint4((uint32_t)o.w0, (uint32_t)(o.w0 >> 32), (uint32_t)o.w1, (uint32_t)(o.w1 >> 32));
                    else
                        reinterpret_cast<uint64_t*>(xflags)[k] = o.w0;
                }
                if (degen) degen[k] = (uint8_t)o.degen;
            }
        } else if (act && r == 0) {
            err |= kDevBadCount;
            if (LOSS) {
                acc += la.scale * w;
                if (la.u_out) la.u_out[k] = 0.f;
            }
            if (!LOSS || iou) iou[k] = 0.f;
            if (SAVE) {
                nx[k] = 0;
                if constexpr (KIN == 8) reinterpret_cast<uint4*>(xflags)[k] = make_uint4(~0u, ~0u, ~0u, ~0u);
                else reinterpret_cast<uint64_t*>(xflags)[k] = ~0ull;
            }
            if (degen) degen[k] = 0;
        }
        if constexpr (DEFER) {
            if (hard && r == 0) iou[k] = __int_as_float(0x7fffffff);
        } else {
            // pairs the group hands back: finished by the whole warp, one at a time
            unsigned todo = __ballot_sync(0xffffffffu, hard && r == 0);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const int64_t kk = base + (src >> 3);
                const int m1 = __shfl_sync(0xffffffffu, n1, src), m2 = __shfl_sync(0xffffffffu, n2, src);
                FwdOut<KIN> o;
                o.err = 0;
                warp_robust<KIN>(p1 + kk * 2 * KIN, p2 + kk * 2 * KIN, m1, m2, refine, o);
                if (lane == src) {
                    if constexpr (Z3) o.iou = iou3_value(o.ai, o.a1, o.a2, o.nx, z_of(za, kk));
                    err |= o.err;
                    put_fwd<KIN, SAVE, LOSS>(o, kk, w, la, iou, nx, xflags, degen, acc);
                }
            }
        }
    }
    if (LOSS) put_partial(la, acc);
    if (err) atomicOr(status, err);
}

// The pairs a deferring forward handed back (IoU marked NaN), finished by
// whole warps in a launch of their own: every warp of this kernel runs the
// warp-cooperative path only, so the SM holds as many of them as its
// registers allow (8 blocks of 128 at 64 registers: measured faster than 5
// or 6) and their long dependent chains overlap.  Warp w scans 32
// IoU values per step (one coalesced load), then takes the marked pairs one
// at a time.  A NaN IoU from NaN inputs is recomputed here too (as NaN).
template <int K, bool SAVE, bool Z3>
__global__ void __launch_bounds__(kPairThreads, 8)
k_paired_fwd_finish(const float* __restrict__ p1, const uint8_t* __restrict__ c1, const float* __restrict__ p2,
                    const uint8_t* __restrict__ c2, int64_t n, float* __restrict__ iou, uint8_t* __restrict__ nx,
                    uint8_t* __restrict__ xflags, uint8_t* __restrict__ degen, uint32_t flags, uint32_t* status,
                    ZArgs za) {
    constexpr unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const bool refine = (flags & kFlagRefine) && !(flags & kFlagPlain);
    const int64_t stride = (int64_t)gridDim.x * kPairThreads;
    const LossArgs la{nullptr, 0.f, nullptr, nullptr, 0};
    uint32_t err = 0;
    float acc = 0.f;
    for (int64_t base = (int64_t)blockIdx.x * kPairThreads + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t k = base + lane;
        const bool mark = k < n && isnan(iou[k]);
        unsigned todo = __ballot_sync(full, mark);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t kk = base + src;
            const int m1 = c1 ? (int)c1[kk] : K, m2 = c2 ? (int)c2[kk] : K;
            FwdOut<K> o;
            o.err = 0;
            warp_robust<K>(p1 + kk * 2 * K, p2 + kk * 2 * K, m1, m2, refine, o);
            if (lane == src) {
                if constexpr (Z3) o.iou = iou3_value(o.ai, o.a1, o.a2, o.nx, z_of(za, kk));
                err |= o.err;
                put_fwd<K, SAVE, false>(o, kk, 0.f, la, iou, nx, xflags, degen, acc);
            }
        }
    }
    if (err) atomicOr(status, err);
}

template <bool RECOMPUTE, bool LOSS, bool Z3, int KIN = 8>
__global__ void __launch_bounds__(kPairThreads, RECOMPUTE ? 1 : kBwdG8MinBlocks)
k_paired_bwd_g8(const float* __restrict__ p1, const uint8_t* __restrict__ c1, const float* __restrict__ p2,
                const uint8_t* __restrict__ c2, int64_t n, const float* __restrict__ grad,
                const uint8_t* __restrict__ nxs, const uint8_t* __restrict__ xflags, float* __restrict__ g1,
                float* __restrict__ g2, uint32_t flags, uint32_t* status, LossArgs la, ZArgs za) {
    constexpr unsigned full = 0xffffffffu;
    __shared__ float s_bwd[kPairThreads / 32][32];
    const int lane = threadIdx.x & 31, r = lane & 7;
    const bool refine = (flags & kFlagRefine) && !(flags & kFlagPlain);
    if constexpr (LOSS) loss_fold(la);
    const int64_t warp = ((int64_t)blockIdx.x * kPairThreads + threadIdx.x) >> 5;
    const int64_t stride = (int64_t)gridDim.x * (kPairThreads / 32) * 4;
    uint32_t err = 0;
    for (int64_t base = warp * 4; base < n; base += stride) {
        const int64_t k = base + (lane >> 3);
        const bool act = k < n;
        const int n1 = (act && c1) ? (int)c1[k] : KIN, n2 = (act && c2) ? (int)c2[k] : KIN;
        const bool good = act && n1 >= 3 && n1 <= KIN && n2 >= 3 && n2 <= KIN;
        bool slow = false, needfwd = false;
        uint64_t w0 = ~0ull, w1 = ~0ull;
        uint32_t nxk = 0;
        float gx1 = 0.f, gy1 = 0.f, gx2 = 0.f, gy2 = 0.f;
        if (good) {
            // the recomputing form needs all of P2 in every lane (the forward's
            // rows); the other takes the lane's own vertices only
            typename std::conditional<RECOMPUTE, g8::Lane, g8::LaneS>::type L;
            if constexpr (RECOMPUTE) g8::load_lane<KIN>(p1 + k * 2 * KIN, p2 + k * 2 * KIN, n1, n2, r, L);
            else g8::load_lane_slim<KIN>(p1 + k * 2 * KIN, p2 + k * 2 * KIN, n1, n2, r, L);
            if constexpr (RECOMPUTE) {
                g8::FwdG o;
                needfwd = refine ? !g8::fwd_group<KIN>(L, o, p1 + k * 2 * KIN, p2 + k * 2 * KIN)
                                 : !g8::fwd_group<KIN>(L, o);
                w0 = o.w0;
                w1 = o.w1;
                nxk = o.nx;
            } else {
                if constexpr (KIN == 8) {
                    const uint4 u = __ldg(reinterpret_cast<const uint4*>(xflags) + k);
                    w0 = (uint64_t)u.x | ((uint64_t)u.y << 32);
                    w1 = (uint64_t)u.z | ((uint64_t)u.w << 32);
                } else {
                    w0 = __ldg(reinterpret_cast<const unsigned long long*>(xflags) + k);
                }
                nxk = nxs[k];
            }
            uint32_t e = kSlow;
            auto adj = make_adj<LOSS, Z3>(la, grad, za, k);
            if (!needfwd) e = g8::bwd_group(L, adj, nxk, w0, w1, refine, gx1, gy1, gx2, gy2);
            slow = e == kSlow;
            if (!slow) {
                if (r == 0) {
                    err |= e;
                    put_zgrad<Z3>(za, k, adj);
                }
                if (r < KIN) {
                    reinterpret_cast<float2*>(g1)[k * KIN + r] = make_float2(gx1, gy1);
                    reinterpret_cast<float2*>(g2)[k * KIN + r] = make_float2(gx2, gy2);
                }
            }
        } else if (act) {
            if (r == 0) {
                err |= kDevBadCount;
                put_zgrad<Z3>(za, k, adj_of<Z3>(0.f, za, k));
            }
            if (r < KIN) {
                reinterpret_cast<float2*>(g1)[k * KIN + r] = make_float2(0.f, 0.f);
                reinterpret_cast<float2*>(g2)[k * KIN + r] = make_float2(0.f, 0.f);
            }
        }
        if (RECOMPUTE) {
            unsigned todo = __ballot_sync(full, needfwd && r == 0);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const int64_t kk = base + (src >> 3);
                const int m1 = __shfl_sync(full, n1, src), m2 = __shfl_sync(full, n2, src);
                FwdOut<KIN> o;
                o.err = 0;
                warp_robust<KIN>(p1 + kk * 2 * KIN, p2 + kk * 2 * KIN, m1, m2, refine, o);
                if (lane == src) {
                    err |= o.err;
                    w0 = o.codes.w[0];
                    if constexpr (KIN == 8) w1 = o.codes.w[1];
                    nxk = o.nx;
                }
            }
        }
        unsigned todo = __ballot_sync(full, slow && r == 0);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t kk = base + (src >> 3);
            const int m1 = __shfl_sync(full, n1, src), m2 = __shfl_sync(full, n2, src);
            const uint32_t mnx = __shfl_sync(full, nxk, src);
            Codes<KIN> cs;
            cs.w[0] = __shfl_sync(full, w0, src);
            if constexpr (KIN == 8) cs.w[1] = __shfl_sync(full, w1, src);
            auto a = make_adj<LOSS, Z3>(la, grad, za, kk);
            const int64_t o2 = kk * 2 * KIN;
            const uint32_t e = refine ? warp_bwd<KIN, ff>(p1 + o2, p2 + o2, m1, m2, a, mnx, cs, g1 + o2, g2 + o2,
                                                          s_bwd[threadIdx.x >> 5])
                                      : warp_bwd<KIN, float>(p1 + o2, p2 + o2, m1, m2, a, mnx, cs, g1 + o2, g2 + o2,
                                                             s_bwd[threadIdx.x >> 5]);
            if (lane == src) {
                err |= e;
                put_zgrad<Z3>(za, kk, a);
            }
        }
    }
    if (err) atomicOr(status, err);
}

} // namespace dgal
