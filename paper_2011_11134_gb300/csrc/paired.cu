// Paired IoU kernels: n independent pairs, one thread per pair.
//
// Forward (paper Sec. II-B `iou`): loads both polygons with 128-bit loads,
// clips in registers (dgal_geom.cuh), stores IoU (4 B), nx (1 B) and the
// 2K code bytes as one 64/128-bit store, plus an optional degeneracy byte.
// Backward (paper Sec. II-B `iou_backward`): reads the polygons, dL/dIoU and
// the recorded (nx, xflags), or recomputes the clip, and writes both
// gradients with 128-bit stores.
#include "dgal_geom.cuh"
#include "dgal_internal.h"
#include "group8.cuh"

namespace dgal {

// One status word per device; every kernel of the library ORs into it through
// a pointer argument (see device_status_ptr in api.cu).
__device__ uint32_t g_status;

uint32_t* status_symbol_address() {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;
    return static_cast<uint32_t*>(p);
}

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

// Both kernels walk the pairs warp by warp (32 consecutive pairs per warp and
// step, grid-stride over warps), with no block-wide barrier.  In the forward,
// a pair the fast path cannot finish (near-degenerate or not in general
// position) is finished afterwards by the whole warp together
// (warp_robust).  In the backward, a pair whose codes the shape derivative
// cannot take (not in general position, or with refinement a tiny
// intersection) runs the shoelace adjoint on its own lane after the rest.

template <int K, bool COUNTS, bool SAVE>
__global__ void __launch_bounds__(kPairThreads)
k_paired_fwd(const float* __restrict__ p1, const uint8_t* __restrict__ c1, const float* __restrict__ p2,
             const uint8_t* __restrict__ c2, int64_t n, float* __restrict__ iou, uint8_t* __restrict__ nx,
             uint8_t* __restrict__ xflags, uint8_t* __restrict__ degen, uint32_t flags, uint32_t* status) {
    constexpr unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * kPairThreads;
    const bool refine = (flags & kFlagRefine) && !(flags & kFlagPlain);
    uint32_t err = 0;
    for (int64_t base = (int64_t)blockIdx.x * kPairThreads + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t k = base + lane;
        int n1 = K, n2 = K;
        bool hard = false;
        if (k < n) {
            if (COUNTS) {
                n1 = c1 ? (int)c1[k] : K;
                n2 = c2 ? (int)c2[k] : K;
            }
            FwdOut<K> o;
            if (COUNTS && (n1 < 3 || n1 > K || n2 < 3 || n2 > K)) {
                err |= kDevBadCount;
                o.nx = 0;
                o.iou = 0.f;
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
                hard = !fwd_generic<K, COUNTS>(g, o);
                if (!hard) {
                    const float U = o.a1 + o.a2 - o.ai;
                    o.iou = (o.nx >= 3u && U > 0.f) ? o.ai / U : 0.f;
                }
            }
            if (!hard) {
                iou[k] = o.iou;
                if (SAVE) {
                    nx[k] = (uint8_t)o.nx;
                    store_codes<K>(xflags, k, o.codes);
                }
                if (degen) degen[k] = (uint8_t)o.degen;
            }
        }
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
                err |= o.err;
                iou[kk] = o.iou;
                if (SAVE) {
                    nx[kk] = (uint8_t)o.nx;
                    store_codes<K>(xflags, kk, o.codes);
                }
                if (degen) degen[kk] = (uint8_t)o.degen;
            }
        }
    }
    if (err) atomicOr(status, err);
}

template <int K, bool COUNTS, bool RECOMPUTE>
__global__ void __launch_bounds__(kPairThreads)
k_paired_bwd(const float* __restrict__ p1, const uint8_t* __restrict__ c1, const float* __restrict__ p2,
             const uint8_t* __restrict__ c2, int64_t n, const float* __restrict__ grad,
             const uint8_t* __restrict__ nxs, const uint8_t* __restrict__ xflags, float* __restrict__ g1,
             float* __restrict__ g2, uint32_t flags, uint32_t* status) {
    constexpr unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * kPairThreads;
    const bool refine = (flags & kFlagRefine) && !(flags & kFlagPlain);
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
                    have = fwd_generic<K, COUNTS>(g, o);
                    codes = o.codes;
                    nxk = o.nx;
                } else {
                    nxk = nxs[k];
                    load_codes<K>(xflags, k, codes);
                }
                uint32_t e = kSlow;
                if (have) e = bwd_shape<K, COUNTS>(g, __ldg(grad + k), nxk, codes, refine, g1x, g1y, g2x, g2y);
                needfwd = !have;
                slow = (e == kSlow);
                if (!slow) err |= e;
            }
            if (!slow) {
                store_poly<K>(g1 + k * 2 * K, g1x, g1y);
                store_poly<K>(g2 + k * 2 * K, g2x, g2y);
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
        if (slow) {
            const float gk = __ldg(grad + k);
            err |= refine ? bwd_shoelace<K, double>(p1 + k * 2 * K, p2 + k * 2 * K, n1, n2, gk, nxk, codes,
                                                    g1 + k * 2 * K, g2 + k * 2 * K)
                          : bwd_shoelace<K, float>(p1 + k * 2 * K, p2 + k * 2 * K, n1, n2, gk, nxk, codes,
                                                   g1 + k * 2 * K, g2 + k * 2 * K);
        }
    }
    if (err) atomicOr(status, err);
}

// K = 8: one group of 8 lanes per pair (group8.cuh), 4 pairs per warp and
// step, grid-stride over warps.  Pairs the group cannot finish are done by the
// whole warp (forward) or by the group's first lane (backward) afterwards.
template <bool SAVE>
__global__ void __launch_bounds__(kPairThreads)
k_paired_fwd_g8(const float* __restrict__ p1, const uint8_t* __restrict__ c1, const float* __restrict__ p2,
                const uint8_t* __restrict__ c2, int64_t n, float* __restrict__ iou, uint8_t* __restrict__ nx,
                uint8_t* __restrict__ xflags, uint8_t* __restrict__ degen, uint32_t flags, uint32_t* status) {
    constexpr unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, r = lane & 7;
    const bool refine = (flags & kFlagRefine) && !(flags & kFlagPlain);
    const int64_t warp = ((int64_t)blockIdx.x * kPairThreads + threadIdx.x) >> 5;
    const int64_t stride = (int64_t)gridDim.x * (kPairThreads / 32) * 4;
    uint32_t err = 0;
    for (int64_t base = warp * 4; base < n; base += stride) {
        const int64_t k = base + (lane >> 3);
        const bool act = k < n;
        const int n1 = (act && c1) ? (int)c1[k] : 8, n2 = (act && c2) ? (int)c2[k] : 8;
        const bool good = act && n1 >= 3 && n1 <= 8 && n2 >= 3 && n2 <= 8;
        bool hard = false;
        if (good) {
            g8::Lane L;
            g8::load_lane(p1 + k * 16, p2 + k * 16, n1, n2, r, L);
            g8::FwdG o;
            hard = !g8::fwd_group(L, o);
            if (!hard && r == 0) {
                iou[k] = o.iou;
                if (SAVE) {
                    nx[k] = (uint8_t)o.nx;
                    reinterpret_cast<uint4*>(xflags)[k] =
                        make_uint4((uint32_t)o.w0, (uint32_t)(o.w0 >> 32), (uint32_t)o.w1, (uint32_t)(o.w1 >> 32));
                }
                if (degen) degen[k] = 0;
            }
        } else if (act && r == 0) {
            err |= kDevBadCount;
            iou[k] = 0.f;
            if (SAVE) {
                nx[k] = 0;
                reinterpret_cast<uint4*>(xflags)[k] = make_uint4(~0u, ~0u, ~0u, ~0u);
            }
            if (degen) degen[k] = 0;
        }
        unsigned todo = __ballot_sync(full, hard && r == 0);
        while (todo) {
            const int src = __ffs(todo) - 1;
            todo &= todo - 1;
            const int64_t kk = base + (src >> 3);
            const int m1 = __shfl_sync(full, n1, src), m2 = __shfl_sync(full, n2, src);
            FwdOut<8> o;
            o.err = 0;
            warp_robust<8>(p1 + kk * 16, p2 + kk * 16, m1, m2, refine, o);
            if (lane == src) {
                err |= o.err;
                iou[kk] = o.iou;
                if (SAVE) {
                    nx[kk] = (uint8_t)o.nx;
                    store_codes<8>(xflags, kk, o.codes);
                }
                if (degen) degen[kk] = (uint8_t)o.degen;
            }
        }
    }
    if (err) atomicOr(status, err);
}

template <bool RECOMPUTE>
__global__ void __launch_bounds__(kPairThreads)
k_paired_bwd_g8(const float* __restrict__ p1, const uint8_t* __restrict__ c1, const float* __restrict__ p2,
                const uint8_t* __restrict__ c2, int64_t n, const float* __restrict__ grad,
                const uint8_t* __restrict__ nxs, const uint8_t* __restrict__ xflags, float* __restrict__ g1,
                float* __restrict__ g2, uint32_t flags, uint32_t* status) {
    constexpr unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, r = lane & 7;
    const bool refine = (flags & kFlagRefine) && !(flags & kFlagPlain);
    const int64_t warp = ((int64_t)blockIdx.x * kPairThreads + threadIdx.x) >> 5;
    const int64_t stride = (int64_t)gridDim.x * (kPairThreads / 32) * 4;
    uint32_t err = 0;
    for (int64_t base = warp * 4; base < n; base += stride) {
        const int64_t k = base + (lane >> 3);
        const bool act = k < n;
        const int n1 = (act && c1) ? (int)c1[k] : 8, n2 = (act && c2) ? (int)c2[k] : 8;
        const bool good = act && n1 >= 3 && n1 <= 8 && n2 >= 3 && n2 <= 8;
        bool slow = false, needfwd = false;
        uint64_t w0 = ~0ull, w1 = ~0ull;
        uint32_t nxk = 0;
        float gx1 = 0.f, gy1 = 0.f, gx2 = 0.f, gy2 = 0.f;
        if (good) {
            g8::Lane L;
            g8::load_lane(p1 + k * 16, p2 + k * 16, n1, n2, r, L);
            if (RECOMPUTE) {
                g8::FwdG o;
                needfwd = !g8::fwd_group(L, o);
                w0 = o.w0;
                w1 = o.w1;
                nxk = o.nx;
            } else {
                const uint4 u = __ldg(reinterpret_cast<const uint4*>(xflags) + k);
                w0 = (uint64_t)u.x | ((uint64_t)u.y << 32);
                w1 = (uint64_t)u.z | ((uint64_t)u.w << 32);
                nxk = nxs[k];
            }
            uint32_t e = kSlow;
            if (!needfwd) e = g8::bwd_group(L, __ldg(grad + k), nxk, w0, w1, refine, gx1, gy1, gx2, gy2);
            slow = e == kSlow;
            if (!slow) {
                if (r == 0) err |= e;
                reinterpret_cast<float2*>(g1)[k * 8 + r] = make_float2(gx1, gy1);
                reinterpret_cast<float2*>(g2)[k * 8 + r] = make_float2(gx2, gy2);
            }
        } else if (act) {
            if (r == 0) err |= kDevBadCount;
            reinterpret_cast<float2*>(g1)[k * 8 + r] = make_float2(0.f, 0.f);
            reinterpret_cast<float2*>(g2)[k * 8 + r] = make_float2(0.f, 0.f);
        }
        if (RECOMPUTE) {
            unsigned todo = __ballot_sync(full, needfwd && r == 0);
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const int64_t kk = base + (src >> 3);
                const int m1 = __shfl_sync(full, n1, src), m2 = __shfl_sync(full, n2, src);
                FwdOut<8> o;
                o.err = 0;
                warp_robust<8>(p1 + kk * 16, p2 + kk * 16, m1, m2, refine, o);
                if (lane == src) {
                    err |= o.err;
                    w0 = o.codes.w[0];
                    w1 = o.codes.w[1];
                    nxk = o.nx;
                }
            }
        }
        if (slow && r == 0) {
            Codes<8> codes;
            codes.w[0] = w0;
            codes.w[1] = w1;
            const float gk = __ldg(grad + k);
            err |= refine ? bwd_shoelace<8, double>(p1 + k * 16, p2 + k * 16, n1, n2, gk, nxk, codes, g1 + k * 16,
                                                    g2 + k * 16)
                          : bwd_shoelace<8, float>(p1 + k * 16, p2 + k * 16, n1, n2, gk, nxk, codes, g1 + k * 16,
                                                   g2 + k * 16);
        }
    }
    if (err) atomicOr(status, err);
}

// ------------------------------------------------------------- fused loss
//
// loss = scale * sum_k w_k (1 - IoU_k) and its gradient in one pass (the
// IoU-loss case study, paper Sec. IV-A): each pair is clipped, its IoU and
// in-register state go straight into the shape-derivative backward with
// dL/dIoU = -scale w_k, and no flags are stored or read back.  Per-thread
// loss terms are reduced per block into partials[blockIdx.x]; a second
// one-block kernel sums the partials in a fixed order (deterministic).

__device__ __forceinline__ float block_sum(float v, float* sh) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    float t = 0.f;
    if (threadIdx.x < 32) {
        t = (l < (int)(blockDim.x >> 5)) ? sh[l] : 0.f;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
    }
    return t;
}

template <bool COUNTS, bool GRADS>
__global__ void __launch_bounds__(kPairThreads)
k_iou_loss4(const float* __restrict__ p1, const uint8_t* __restrict__ c1, const float* __restrict__ p2,
            const uint8_t* __restrict__ c2, int64_t n, const float* __restrict__ weight, float scale,
            float* __restrict__ iou, float* __restrict__ g1, float* __restrict__ g2, float* __restrict__ partials,
            uint32_t flags, uint32_t* status) {
    constexpr int K = 4;
    constexpr unsigned full = 0xffffffffu;
    __shared__ float sh[kPairThreads / 32];
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * kPairThreads;
    const bool refine = (flags & kFlagRefine) && !(flags & kFlagPlain);
    uint32_t err = 0;
    float acc = 0.f;
    for (int64_t base = (int64_t)blockIdx.x * kPairThreads + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t k = base + lane;
        int n1 = K, n2 = K;
        bool hard = false, slow = false;
        float w = 0.f, iv = 0.f;
        Codes<K> codes;
        codes_fill<K>(codes, ~0ull);
        uint32_t nxk = 0;
        if (k < n) {
            if (COUNTS) {
                n1 = c1 ? (int)c1[k] : K;
                n2 = c2 ? (int)c2[k] : K;
            }
            w = weight ? __ldg(weight + k) : 1.f;
            float gx1[K], gy1[K], gx2[K], gy2[K];
#pragma unroll
            for (int v = 0; v < K; ++v) { gx1[v] = gy1[v] = gx2[v] = gy2[v] = 0.f; }
            if (COUNTS && (n1 < 3 || n1 > K || n2 < 3 || n2 > K)) {
                err |= kDevBadCount;
            } else {
                float px[K], py[K], qx[K], qy[K];
                load_poly<K>(p1 + k * 2 * K, px, py);
                load_poly<K>(p2 + k * 2 * K, qx, qy);
                Geo<K> g;
                make_geo<K, COUNTS>(px, py, qx, qy, n1, n2, g);
                FwdOut<K> o;
                input_areas<K, COUNTS>(g, o.a1, o.a2);
                hard = !fwd_generic<K, COUNTS>(g, o);
                if (!hard) {
                    const float U = o.a1 + o.a2 - o.ai;
                    iv = (o.nx >= 3u && U > 0.f) ? o.ai / U : 0.f;
                    if (GRADS) {
                        const uint32_t e = bwd_shape<K, COUNTS>(g, -scale * w, o.nx, o.codes, refine, gx1, gy1, gx2, gy2);
                        slow = e == kSlow;
                        if (!slow) err |= e;
                        codes = o.codes;
                        nxk = o.nx;
                    }
                }
            }
            if (!hard) {
                acc += scale * w * (1.f - iv);
                if (iou) iou[k] = iv;
                if (GRADS && !slow) {
                    store_poly<K>(g1 + k * 2 * K, gx1, gy1);
                    store_poly<K>(g2 + k * 2 * K, gx2, gy2);
                }
            }
        }
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
                err |= o.err;
                iv = o.iou;
                codes = o.codes;
                nxk = o.nx;
                acc += scale * w * (1.f - iv);
                if (iou) iou[kk] = iv;
                slow = true;
            }
        }
        if (GRADS && slow) {
            err |= refine ? bwd_shoelace<K, double>(p1 + k * 2 * K, p2 + k * 2 * K, n1, n2, -scale * w, nxk, codes,
                                                    g1 + k * 2 * K, g2 + k * 2 * K)
                          : bwd_shoelace<K, float>(p1 + k * 2 * K, p2 + k * 2 * K, n1, n2, -scale * w, nxk, codes,
                                                   g1 + k * 2 * K, g2 + k * 2 * K);
        }
    }
    const float tot = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = tot;
    if (err) atomicOr(status, err);
}

__global__ void __launch_bounds__(1024) k_sum_partials(const float* __restrict__ partials, int m, float* __restrict__ out) {
    __shared__ float sh[32];
    float v = 0.f;
    for (int i = threadIdx.x; i < m; i += blockDim.x) v += partials[i];
    const float t = block_sum(v, sh);
    if (threadIdx.x == 0) *out = t;
}

static unsigned grid_for(int64_t n, int threads) {
    int64_t blocks = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count() * 64;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (unsigned)blocks;
}

template <int K, bool COUNTS>
static void fwd_dispatch(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                         float* iou, uint8_t* nx, uint8_t* xflags, uint8_t* degen, uint32_t flags, cudaStream_t s) {
    const unsigned grid = grid_for(n, kPairThreads);
    uint32_t* st = device_status_ptr();
    if (nx) k_paired_fwd<K, COUNTS, true><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st);
    else k_paired_fwd<K, COUNTS, false><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st);
}

dgal_status launch_paired_fwd(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                              int K, float* iou, uint8_t* nx, uint8_t* xflags, uint8_t* degen, uint32_t flags,
                              cudaStream_t s) {
    if (!device_status_ptr()) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    const bool counts = c1 || c2;
    if (K == 4) {
        if (counts) fwd_dispatch<4, true>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, s);
        else fwd_dispatch<4, false>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, s);
    } else {
        const unsigned grid = grid_for((n + 3) / 4 * 32, kPairThreads);
        uint32_t* st = device_status_ptr();
        if (nx) k_paired_fwd_g8<true><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st);
        else k_paired_fwd_g8<false><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st);
    }
    return check_launch("paired forward");
}

template <int K, bool COUNTS>
static void bwd_dispatch(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                         const float* grad, const uint8_t* nx, const uint8_t* xflags, float* g1, float* g2,
                         uint32_t flags, cudaStream_t s) {
    const unsigned grid = grid_for(n, kPairThreads);
    uint32_t* st = device_status_ptr();
    if (nx && xflags && !(flags & kFlagPlain))
        k_paired_bwd<K, COUNTS, false><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, st);
    else
        k_paired_bwd<K, COUNTS, true><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, st);
}

dgal_status launch_paired_bwd(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                              int K, const float* grad, const uint8_t* nx, const uint8_t* xflags, float* g1,
                              float* g2, uint32_t flags, cudaStream_t s) {
    if (!device_status_ptr()) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    const bool counts = c1 || c2;
    if (K == 4) {
        if (counts) bwd_dispatch<4, true>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, s);
        else bwd_dispatch<4, false>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, s);
    } else {
        const unsigned grid = grid_for((n + 3) / 4 * 32, kPairThreads);
        uint32_t* st = device_status_ptr();
        if (nx && xflags && !(flags & kFlagPlain))
            k_paired_bwd_g8<false><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, st);
        else
            k_paired_bwd_g8<true><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, st);
    }
    return check_launch("paired backward");
}

size_t loss_workspace_bytes(int64_t n) {
    const int64_t blocks = (int64_t)grid_for(n < 1 ? 1 : n, kPairThreads);
    return (size_t)(((blocks * 4) + 255) / 256 * 256);
}

dgal_status launch_iou_loss(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n, int K,
                            const float* weight, float scale, float* loss, float* iou, float* g1, float* g2,
                            void* ws, uint32_t flags, cudaStream_t s) {
    if (!device_status_ptr()) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    const unsigned grid = grid_for(n, kPairThreads);
    float* partials = static_cast<float*>(ws);
    uint32_t* st = device_status_ptr();
    const bool counts = c1 || c2;
    if (K != 4) return fail(DGAL_ERR_UNSUPPORTED_K, "the fused loss supports K = 4");
    if (counts) {
        if (g1) k_iou_loss4<true, true><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, weight, scale, iou, g1, g2, partials, flags, st);
        else k_iou_loss4<true, false><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, weight, scale, iou, g1, g2, partials, flags, st);
    } else {
        if (g1) k_iou_loss4<false, true><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, weight, scale, iou, g1, g2, partials, flags, st);
        else k_iou_loss4<false, false><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, weight, scale, iou, g1, g2, partials, flags, st);
    }
    dgal_status r = check_launch("fused IoU loss");
    if (r != DGAL_OK) return r;
    k_sum_partials<<<1, 1024, 0, s>>>(partials, (int)grid, loss);
    return check_launch("fused IoU loss reduction");
}

} // namespace dgal
