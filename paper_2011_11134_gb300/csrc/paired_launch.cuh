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
// lanes per pair for K = 8.  The group kernels loop over at most 256 blocks
// per SM (measured against 64 and 2048 on the 4M-pair convex step: 2.17,
// 2.13 and 2.22 ms).
static unsigned paired_grid(int64_t n, int K) {
    if (K == 4) return grid_for(n, kPairThreads);
    int64_t blocks = ((n + 3) / 4 * 32 + kPairThreads - 1) / kPairThreads;
    const int64_t cap = (int64_t)sm_count() * 256;
    if (blocks > cap) blocks = cap;
    return (unsigned)(blocks < 1 ? 1 : blocks);
}

template <int K, bool COUNTS, bool LOSS, bool Z3>
static void fwd_dispatch(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                         float* iou, uint8_t* nx, uint8_t* xflags, uint8_t* degen, uint32_t flags, cudaStream_t s,
                         const LossArgs& la, const ZArgs& za, int64_t n_shape = -1) {
    const unsigned grid = paired_grid(n, K);
    uint32_t* st = device_status_ptr();
    if constexpr (K == 4 && !LOSS) {
        // n_shape: the batch size that picks the launch shape (a chunk of a
        // larger batch takes the whole batch's shape, so results match)
        if ((n_shape >= 0 ? n_shape : n) < paired_config(4).group_below) {
            // a small batch: a group of 8 lanes per quadrilateral pair
            const unsigned ggrid = paired_grid(n, 8);
            if (nx) k_paired_fwd_g8<true, false, Z3, false, 4><<<ggrid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st, la, za);
            else k_paired_fwd_g8<false, false, Z3, false, 4><<<ggrid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st, la, za);
            return;
        }
    }
    if constexpr (K == 4) {
        if (nx) k_paired_fwd<K, COUNTS, true, LOSS, Z3><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st, la, za);
        else k_paired_fwd<K, COUNTS, false, LOSS, Z3><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st, la, za);
    } else {
        if constexpr (!LOSS) {
            // hard pairs finished by a second launch sized for the warp path
            const unsigned fgrid = grid_for(n, kPairThreads);
            if (nx) {
                k_paired_fwd_g8<true, false, Z3, true><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st, la, za);
                k_paired_fwd_finish<8, true, Z3><<<fgrid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st, za);
            } else {
                k_paired_fwd_g8<false, false, Z3, true><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st, la, za);
                k_paired_fwd_finish<8, false, Z3><<<fgrid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st, za);
            }
        } else {
            if (nx) k_paired_fwd_g8<true, LOSS, Z3><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st, la, za);
            else k_paired_fwd_g8<false, LOSS, Z3><<<grid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, st, la, za);
        }
    }
}

// Forward for K = 4 or 8; Z3 selects the 3D IoU.
template <bool LOSS, bool Z3>
static void fwd_any(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n, int K,
                    float* iou, uint8_t* nx, uint8_t* xflags, uint8_t* degen, uint32_t flags, cudaStream_t s,
                    const LossArgs& la, const ZArgs& za, int64_t n_shape = -1) {
    if (K == 4) {
        if (c1 || c2) fwd_dispatch<4, true, LOSS, Z3>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, s, la, za, n_shape);
        else fwd_dispatch<4, false, LOSS, Z3>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, s, la, za, n_shape);
    } else {
        fwd_dispatch<8, true, LOSS, Z3>(p1, c1, p2, c2, n, iou, nx, xflags, degen, flags, s, la, za);
    }
}

// Launches kernel k with programmatic stream serialisation: its blocks may
// be scheduled while the kernel before it in the stream is finishing (the
// paired forward lets them start with griddepcontrol.launch_dependents), so
// the backward's launch and block scheduling overlap the forward's last wave.
// The kernel itself waits for the previous grid (griddepcontrol.wait) before
// it touches memory.  Measured on the 1M-pair step: 74.1 -> 71.7 us.  If the
// runtime refuses the attribute, the same kernel is launched the plain way.
template <typename... P, typename... A>
static void launch_pdl(void (*kern)(P...), unsigned grid, unsigned block, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    if (cudaLaunchKernelEx(&cfg, kern, args...) != cudaSuccess) {
        (void)cudaGetLastError();
        kern<<<grid, block, 0, s>>>(args...);
    }
}

template <int K, bool COUNTS, bool LOSS, bool Z3>
static void bwd_dispatch(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                         const float* grad, const uint8_t* nx, const uint8_t* xflags, float* g1, float* g2,
                         uint32_t flags, cudaStream_t s, const LossArgs& la, const ZArgs& za, int64_t n_shape = -1) {
    const unsigned grid = paired_grid(n, K);
    uint32_t* st = device_status_ptr();
    const bool saved = nx && xflags && !(flags & kFlagPlain);
    if constexpr (K == 4 && !LOSS) {
        if ((n_shape >= 0 ? n_shape : n) < paired_config(4).group_below) {
            const unsigned ggrid = paired_grid(n, 8);
            if (saved)
                k_paired_bwd_g8<false, false, Z3, 4><<<ggrid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, st, la, za);
            else
                k_paired_bwd_g8<true, false, Z3, 4><<<ggrid, kPairThreads, 0, s>>>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, st, la, za);
            return;
        }
    }
    if constexpr (K == 4) {
        if (saved)
            launch_pdl(k_paired_bwd<K, COUNTS, false, LOSS, Z3>, grid, kPairThreads, s, p1, c1, p2, c2, n, grad, nx,
                       xflags, g1, g2, flags, st, la, za);
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
                    uint32_t flags, cudaStream_t s, const LossArgs& la, const ZArgs& za, int64_t n_shape = -1) {
    if (K == 4) {
        if (c1 || c2) bwd_dispatch<4, true, LOSS, Z3>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, s, la, za, n_shape);
        else bwd_dispatch<4, false, LOSS, Z3>(p1, c1, p2, c2, n, grad, nx, xflags, g1, g2, flags, s, la, za, n_shape);
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

// Loss workspace: [per-warp partials | partials of the GIoU / DIoU terms |
// U per pair | A_h per pair | GIoU hull order and count (16 bytes a pair) |
// nx (n bytes) | xflags (n x 2K bytes)], each
// part 256-byte aligned.
struct LossLayout {
    size_t partials, partials2, u, ah, aux, nx, xflags, total;
    int64_t warps, warps2;
};

static LossLayout loss_layout(int64_t n, int K) {
    auto up = [](size_t b) { return (b + 255) / 256 * 256; };
    LossLayout L;
    // one partial per warp of the forward grid, and of the GIoU / DIoU pass
    L.warps = (int64_t)paired_grid(n < 1 ? 1 : n, K) * (kPairThreads / 32);
    L.warps2 = loss_var_partials(n < 1 ? 1 : n);
    L.partials = 0;
    L.partials2 = up((size_t)L.warps * 4);
    L.u = L.partials2 + up((size_t)L.warps2 * 4);
    L.ah = L.u + up((size_t)n * 4);
    L.aux = L.ah + up((size_t)n * 4);
    L.nx = L.aux + up((size_t)n * 16);
    L.xflags = L.nx + up((size_t)n);
    L.total = L.xflags + up((size_t)n * 2 * K);
    return L;
}

// 0: the IoU loss, 1: GIoU, 2: DIoU (from the flag bits).
static int loss_variant(uint32_t flags) {
    return (flags & DGAL_LOSS_GIOU) ? 1 : (flags & DGAL_LOSS_DIOU) ? 2 : 0;
}

// The loss forward: the paired forward in loss mode (flags kept in the
// workspace unless DGAL_PLAIN; U kept for the GIoU / DIoU terms), then the
// GIoU / DIoU pass.  With `fold`, the partials are summed into loss[0] here
// (a one-block launch); otherwise the backward's block 0 sums them.
template <bool Z3>
static dgal_status iou_loss_forward(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                                    int K, const float* weight, float scale, float* loss, float* iou,
                                    const ZArgs& za, void* ws, uint32_t flags, bool fold, cudaStream_t s) {
    const LossLayout L = loss_layout(n, K);
    const int var = loss_variant(flags);
    unsigned char* base = static_cast<unsigned char*>(ws);
    LossArgs la{weight, scale, reinterpret_cast<float*>(base + L.partials), nullptr, 0};
    if (var) la.u_out = reinterpret_cast<float*>(base + L.u);
    const bool save = !(flags & kFlagPlain);
    fwd_any<true, Z3>(p1, c1, p2, c2, n, K, iou, save ? base + L.nx : nullptr, save ? base + L.xflags : nullptr,
                      nullptr, flags, s, la, za);
    dgal_status r = check_launch("IoU loss forward");
    if (r != DGAL_OK) return r;
    float* partials2 = reinterpret_cast<float*>(base + L.partials2);
    if (var) {
        r = launch_loss_var_fwd(var, p1, c1, p2, c2, n, K, weight, scale, la.u_out,
                                reinterpret_cast<float*>(base + L.ah), reinterpret_cast<uint64_t*>(base + L.aux),
                                partials2, s);
        if (r != DGAL_OK) return r;
    }
    if (!fold) return DGAL_OK;
    launch_sum_partials(la.partials, L.warps, var ? partials2 : nullptr, L.warps2, loss, s);
    return check_launch("IoU loss reduction");
}

// The loss backward from the state a forward left in the workspace: the
// paired backward in loss mode (reading the saved flags, or recomputing the
// clip under DGAL_PLAIN), its block 0 summing the partials into loss[0] when
// loss is set, then the GIoU / DIoU gradient pass.  dloss: device pointer to
// the upstream gradient of the loss, or NULL for 1.
template <bool Z3>
static dgal_status iou_loss_backward(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2,
                                     int64_t n, int K, const float* weight, float scale, const float* dloss, float* loss,
                                     float* g1, float* g2, const ZArgs& za, void* ws, uint32_t flags, cudaStream_t s) {
    const LossLayout L = loss_layout(n, K);
    const int var = loss_variant(flags);
    unsigned char* base = static_cast<unsigned char*>(ws);
    const bool save = !(flags & kFlagPlain);
    LossArgs lb{weight, scale, reinterpret_cast<float*>(base + L.partials), loss, L.warps};
    lb.dloss = dloss;
    if (var) {
        lb.partials2 = reinterpret_cast<const float*>(base + L.partials2);
        lb.nparts2 = L.warps2;
    }
    if (var == 1) lb.ah = reinterpret_cast<const float*>(base + L.ah);
    bwd_any<true, Z3>(p1, c1, p2, c2, n, K, nullptr, save ? base + L.nx : nullptr, save ? base + L.xflags : nullptr,
                      g1, g2, flags, s, lb, za);
    dgal_status r = check_launch("IoU loss backward");
    if (r != DGAL_OK || !var) return r;
    return launch_loss_var_bwd(var, p1, c1, p2, c2, n, K, weight, scale, dloss,
                               reinterpret_cast<const float*>(base + L.u), reinterpret_cast<const float*>(base + L.ah),
                               reinterpret_cast<const uint64_t*>(base + L.aux), g1, g2, s);
}

// The loss and (when g1 is set) its gradient in one call.
template <bool Z3>
static dgal_status iou_loss_passes(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                                   int K, const float* weight, float scale, float* loss, float* iou, float* g1,
                                   float* g2, const ZArgs& za, void* ws, uint32_t flags, cudaStream_t s) {
    dgal_status r = iou_loss_forward<Z3>(p1, c1, p2, c2, n, K, weight, scale, loss, iou, za, ws, flags, !g1, s);
    if (r != DGAL_OK || !g1) return r;
    return iou_loss_backward<Z3>(p1, c1, p2, c2, n, K, weight, scale, nullptr, loss, g1, g2, za, ws, flags, s);
}

} // namespace dgal
