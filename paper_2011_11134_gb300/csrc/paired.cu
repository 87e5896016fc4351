// Paired IoU kernels: n independent pairs, one thread per pair.
//
// Forward (paper Sec. II-B `iou`): loads both polygons with 128-bit loads,
// clips in registers (dgal_geom.cuh), stores IoU (4 B), nx (1 B) and the
// 2K code bytes as one 64/128-bit store, plus an optional degeneracy byte.
// Backward (paper Sec. II-B `iou_backward`): reads the polygons, dL/dIoU and
// the recorded (nx, xflags), or recomputes the clip, and writes both
// gradients with 128-bit stores.
#include "paired_launch.cuh"

namespace dgal {

// One status word per device; every kernel of the library ORs into it through
// a pointer argument (see device_status_ptr in api.cu).
__device__ uint32_t g_status;

uint32_t* status_symbol_address() {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_status) != cudaSuccess) return nullptr;
    return static_cast<uint32_t*>(p);
}

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

// One block sums the m per-warp loss partials in a fixed order (then the m2
// partials of the GIoU / DIoU terms, when given): fold_part's rounds over each
// array, then a fixed tree.  The order does not depend on scheduling, so the
// loss is deterministic.  The partials must be 16-byte aligned.
constexpr int kSumThreads = 1024;

__global__ void __launch_bounds__(kSumThreads) k_sum_partials(const float* __restrict__ partials, int64_t m,
                                                               const float* __restrict__ partials2, int64_t m2,
                                                               float* __restrict__ out) {
    __shared__ float sh[32];
    float v = fold_part(partials, m);
    if (partials2) v += fold_part(partials2, m2);
    const float t = block_sum(v, sh);
    if (threadIdx.x == 0) *out = t;
}

void launch_sum_partials(const float* partials, int64_t m, const float* partials2, int64_t m2, float* out,
                         cudaStream_t s) {
    k_sum_partials<<<1, kSumThreads, 0, s>>>(partials, m, partials2, m2, out);
}

dgal_status launch_paired_fwd(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                              int K, float* iou, uint8_t* nx, uint8_t* xflags, uint8_t* degen, uint32_t flags,
                              cudaStream_t s, int64_t n_shape) {
    if (!device_status_ptr()) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    fwd_any<false, false>(p1, c1, p2, c2, n, K, iou, nx, xflags, degen, flags, s, LossArgs{nullptr, 0.f, nullptr},
                          ZArgs{nullptr, nullptr, nullptr, nullptr}, n_shape);
    return check_launch("paired forward");
}

dgal_status launch_paired_bwd(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                              int K, const float* grad, const uint8_t* nx, const uint8_t* xflags, float* g1,
                              float* g2, uint32_t flags, cudaStream_t s, int64_t n_shape) {
    if (!device_status_ptr()) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    bwd_any<false, false>(p1, c1, p2, c2, n, K, grad, nx, xflags, g1, g2, flags, s, LossArgs{nullptr, 0.f, nullptr},
                          ZArgs{nullptr, nullptr, nullptr, nullptr}, n_shape);
    return check_launch("paired backward");
}

dgal_status launch_paired_fused(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                                int K, const float* grad, float* iou, float* g1, float* g2, uint32_t flags,
                                cudaStream_t s) {
    uint32_t* st = device_status_ptr();
    if (!st) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    if (K != 4) return fail(DGAL_ERR_UNSUPPORTED_K, "the one-pass form takes K = 4");
    const unsigned grid = paired_grid(n, K);
    if (c1 || c2)
        k_paired_fused<4, true><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, grad, iou, g1, g2, flags, st);
    else
        k_paired_fused<4, false><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, grad, iou, g1, g2, flags, st);
    return check_launch("paired forward + backward");
}

size_t loss_workspace_bytes(int64_t n, int K) { return loss_layout(n, K).total; }

dgal_status launch_iou_loss(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n, int K,
                            const float* weight, float scale, float* loss, float* iou, float* g1, float* g2,
                            void* ws, uint32_t flags, cudaStream_t s) {
    if (!device_status_ptr()) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    return iou_loss_passes<false>(p1, c1, p2, c2, n, K, weight, scale, loss, iou, g1, g2,
                                  ZArgs{nullptr, nullptr, nullptr, nullptr}, ws, flags, s);
}

dgal_status launch_iou_loss_backward(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                                     int K, const float* weight, float scale, const float* dloss, float* g1,
                                     float* g2, void* ws, uint32_t flags, cudaStream_t s) {
    if (!device_status_ptr()) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    return iou_loss_backward<false>(p1, c1, p2, c2, n, K, weight, scale, dloss, nullptr, g1, g2,
                                    ZArgs{nullptr, nullptr, nullptr, nullptr}, ws, flags, s);
}

} // namespace dgal
