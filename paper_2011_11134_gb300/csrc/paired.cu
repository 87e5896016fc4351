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
        if (counts) fwd_dispatch<8, true>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, s);
        else fwd_dispatch<8, false>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, s);
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
        if (counts) bwd_dispatch<8, true>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, s);
        else bwd_dispatch<8, false>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, s);
    }
    return check_launch("paired backward");
}

} // namespace dgal
