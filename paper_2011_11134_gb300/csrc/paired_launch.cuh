// Launch configuration and dispatch of the paired kernels (included by
// paired.cu for the 2D IoU and by paired3d.cu for the 3D IoU): one thread per
// pair for K = 4, one group of 8 lanes per pair for K = 8
// (paired_kernels.cuh).
#pragma once

#include "paired_kernels.cuh"

namespace dgal {

static unsigned grid_for(int64_t n, int threads) {
    int64_t blocks = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count() * 64;
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    return (unsigned)blocks;
}

// Grid of the paired kernels: one thread per pair for K = 4, one group of 8
// lanes per pair for K = 8.
static unsigned paired_grid(int64_t n, int K) {
    return K == 4 ? grid_for(n, kPairThreads) : grid_for((n + 3) / 4 * 32, kPairThreads);
}

template <int K, bool COUNTS, bool LOSS, bool Z3>
static void fwd_dispatch(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                         float* iou, uint8_t* nx, uint8_t* xflags, uint8_t* degen, uint32_t flags, cudaStream_t s,
                         const LossArgs& la, const ZArgs& za) {
    const unsigned grid = paired_grid(n, K);
    uint32_t* st = device_status_ptr();
    if constexpr (K == 4) {
        if (nx) k_paired_fwd<K, COUNTS, true, LOSS, Z3><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st, la, za);
        else k_paired_fwd<K, COUNTS, false, LOSS, Z3><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st, la, za);
    } else {
        if (nx) k_paired_fwd_g8<true, LOSS, Z3><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st, la, za);
        else k_paired_fwd_g8<false, LOSS, Z3><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st, la, za);
    }
}

// Forward for K = 4 or 8; Z3 selects the 3D IoU.
template <bool LOSS, bool Z3>
static void fwd_any(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n, int K,
                    float* iou, uint8_t* nx, uint8_t* xflags, uint8_t* degen, uint32_t flags, cudaStream_t s,
                    const LossArgs& la, const ZArgs& za) {
    if (K == 4) {
        if (c1 || c2) fwd_dispatch<4, true, LOSS, Z3>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, s, la, za);
        else fwd_dispatch<4, false, LOSS, Z3>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, s, la, za);
    } else {
        fwd_dispatch<8, true, LOSS, Z3>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, s, la, za);
    }
}

template <int K, bool COUNTS, bool LOSS, bool Z3>
static void bwd_dispatch(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                         const float* grad, const uint8_t* nx, const uint8_t* xflags, float* g1, float* g2,
                         uint32_t flags, cudaStream_t s, const LossArgs& la, const ZArgs& za) {
    const unsigned grid = paired_grid(n, K);
    uint32_t* st = device_status_ptr();
    const bool saved = nx && xflags && !(flags & kFlagPlain);
    if constexpr (K == 4) {
        if (saved)
            k_paired_bwd<K, COUNTS, false, LOSS, Z3><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, st, la, za);
        else
            k_paired_bwd<K, COUNTS, true, LOSS, Z3><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, st, la, za);
    } else {
        if (saved)
            k_paired_bwd_g8<false, LOSS, Z3><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, st, la, za);
        else
            k_paired_bwd_g8<true, LOSS, Z3><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, st, la, za);
    }
}

template <bool LOSS, bool Z3>
static void bwd_any(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n, int K,
                    const float* grad, const uint8_t* nx, const uint8_t* xflags, float* g1, float* g2,
                    uint32_t flags, cudaStream_t s, const LossArgs& la, const ZArgs& za) {
    if (K == 4) {
        if (c1 || c2) bwd_dispatch<4, true, LOSS, Z3>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, s, la, za);
        else bwd_dispatch<4, false, LOSS, Z3>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, s, la, za);
    } else {
        bwd_dispatch<8, true, LOSS, Z3>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, s, la, za);
    }
}

// ------------------------------------------------------------- IoU loss
//
// loss = scale * sum_k w_k (1 - IoU_k) and its gradient (the IoU-loss case
// study, paper Sec. IV-A) in two launches on one stream: the paired forward
// in loss mode (no IoU array needed; flags saved to the workspace) and the
// paired backward in loss mode (dL/dIoU formed in the kernel), whose block 0
// also sums the per-warp partials in a fixed order (loss_fold), so the loss
// is deterministic.  A single kernel doing both passes was measured slower:
// with the forward and backward code resident together it needs about 1.5x
// the registers and stalls on instruction fetch.

// Loss workspace: [per-warp partials | nx (n bytes) | xflags (n x 2K bytes)],
// each part 256-byte aligned.
struct LossLayout {
    size_t partials, nx, xflags, total;
    int64_t warps;
};

static LossLayout loss_layout(int64_t n, int K) {
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    LossLayout L;
    // one partial per warp of the forward grid
    L.warps = (int64_t)paired_grid(n < 1 ? 1 : n, K) * (kPairThreads / 32);
    L.partials = 0;
    L.nx = up((size_t)L.warps * 4);
    L.xflags = L.nx + up((size_t)n);
    L.total = L.xflags + up((size_t)n * 2 * K);
    return L;
}

// The loss passes: the forward in loss mode, then the backward in loss mode
// with the partial sum folded into its block 0, or (no gradients wanted) the
// one-block partial sum on its own.
template <bool Z3>
static dgal_status iou_loss_passes(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                                   int K, const float* weight, float scale, float* loss, float* iou, float* g1,
                                   float* g2, const ZArgs& za, void* ws, uint32_t flags, cudaStream_t s) {
    const LossLayout L = loss_layout(n, K);
    const int64_t nparts = L.warps; // one partial per warp of the forward grid
    unsigned char* base = static_cast<unsigned char*>(ws);
    const LossArgs la{weight, scale, reinterpret_cast<float*>(base + L.partials), nullptr, 0};
    const bool save = g1 && !(flags & kFlagPlain);
    uint8_t* nx = base + L.nx;
    uint8_t* xflags = base + L.xflags;
    fwd_any<true, Z3>(p1, c1, p2, c2, n, K, iou, nx, xflags, nullptr, flags, s, la, za);
    dgal_status r = check_launch("IoU loss forward");
    if (r != DGAL_OK) return r;
    if (g1) {
        const LossArgs lb{weight, scale, la.partials, loss, nparts};
        bwd_any<true, Z3>(p1, c1, p2, c2, n, K, nullptr, save ? nx : nullptr, save ? xflags : nullptr, g1, g2, flags,
                          s, lb, za);
        return check_launch("IoU loss backward");
    }
    launch_sum_partials(la.partials, nparts, loss, s);
    return check_launch("IoU loss reduction");
}

} // namespace dgal
