// Internal host-side declarations shared by the libdgal translation units.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "dgal.h"

namespace dgal {

// Records a message for dgal_last_error() and returns `st`.
dgal_status fail(dgal_status st, const char* fmt, ...);
// Clears the calling host thread's dgal_last_error() message.
void clear_last_error();
// Argument checks of the ragged batch that do not involve its workspace (K,
// S, offset / polygon / output pointers and their alignment).
dgal_status check_batched_args(int S, const int64_t* a_off, const int64_t* b_off, const int64_t* out_off,
                               const float* a, const float* b, int K, const float* iou);
// Checks cudaGetLastError after a launch.
dgal_status check_launch(const char* what);
// Number of SMs of the current device (cached per device).
int sm_count();
// Address of the device status word on the current device (cached per device).
uint32_t* device_status_ptr();
// Uncached lookup of that address (paired.cu owns the symbol).
uint32_t* status_symbol_address();

// Launch shape of the ragged batched kernel.
struct BatchedConfig {
    int tile;       // entries per tile (one queue pop)
    int threads;    // threads per block
    int blocks_sm;  // resident blocks per SM of the persistent grid
};
BatchedConfig batched_config(int K);
void set_batched_config(int K, BatchedConfig c);

// Launch shape of the paired kernels for quadrilaterals: below group_below
// pairs a group of 8 lanes takes each pair (lower latency for small
// batches), from there one lane per pair (fewer instructions per pair).
struct PairedConfig {
    int64_t group_below;
};
PairedConfig paired_config(int K);
void set_paired_config(int K, PairedConfig c);

// Launchers (no validation; called from the C ABI after checks).
// n_shape: the batch size that picks the launch shape (default n; a chunk of
// a larger batch passes the whole batch's size so that results match).
// DGAL_VALIDATE / dgal_validate_polygons: the convexity and orientation check
// of n polygons (geom_ops.cu); bad (nullable) receives 1 per failing polygon.
dgal_status launch_validate(const float* p, const uint8_t* c, int64_t n, int K, uint8_t* bad, cudaStream_t s);
dgal_status launch_paired_fwd(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                              int K, float* iou, uint8_t* nx, uint8_t* xflags, uint8_t* degen, uint32_t flags,
                              cudaStream_t s, int64_t n_shape = -1);
dgal_status launch_paired_bwd(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                              int K, const float* grad, const uint8_t* nx, const uint8_t* xflags, float* g1,
                              float* g2, uint32_t flags, cudaStream_t s, int64_t n_shape = -1);
// K = 4: forward + backward in one pass (pointers may be device-mapped host memory).
dgal_status launch_paired_fused(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                                int K, const float* grad, float* iou, float* g1, float* g2, uint32_t flags,
                                cudaStream_t s);
dgal_status launch_pairwise(const float* a, const uint8_t* ca, int64_t N, const float* b, const uint8_t* cb,
                            int64_t M, int K, float* iou, uint8_t* nx, uint32_t flags, cudaStream_t s);
size_t batched_workspace_bytes(int S);
size_t loss_workspace_bytes(int64_t n, int K);
dgal_status launch_iou_loss(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n, int K,
                            const float* weight, float scale, float* loss, float* iou, float* g1, float* g2,
                            void* ws, uint32_t flags, cudaStream_t s);
// 3D IoU (z1 / z2: float [n][2] = (z_center, height)) and its backward,
// paired3d.cu.
dgal_status launch_paired3d_fwd(const float* p1, const uint8_t* c1, const float* z1, const float* p2,
                                const uint8_t* c2, const float* z2, int64_t n, int K, float* iou, uint8_t* nx,
                                uint8_t* xflags, uint8_t* degen, uint32_t flags, cudaStream_t s);
dgal_status launch_paired3d_bwd(const float* p1, const uint8_t* c1, const float* z1, const float* p2,
                                const uint8_t* c2, const float* z2, int64_t n, int K, const float* grad,
                                const uint8_t* nx, const uint8_t* xflags, float* g1, float* gz1, float* g2, float* gz2,
                                uint32_t flags, cudaStream_t s);
dgal_status launch_iou3d_loss(const float* p1, const uint8_t* c1, const float* z1, const float* p2, const uint8_t* c2,
                              const float* z2, int64_t n, int K, const float* weight, float scale, float* loss,
                              float* iou, float* g1, float* gz1, float* g2, float* gz2, void* ws, uint32_t flags,
                              cudaStream_t s);
// One-block fixed-order sum of m per-warp loss partials (and of m2 more from
// partials2 when it is not NULL) into *out.
void launch_sum_partials(const float* partials, int64_t m, const float* partials2, int64_t m2, float* out,
                         cudaStream_t s);
// Backward of the IoU loss from the state a forward-only dgal_iou_loss left
// in the workspace; dloss: device pointer to the loss's upstream gradient.
dgal_status launch_iou_loss_backward(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                                     int K, const float* weight, float scale, const float* dloss, float* g1,
                                     float* g2, void* ws, uint32_t flags, cudaStream_t s);
dgal_status launch_iou3d_loss_backward(const float* p1, const uint8_t* c1, const float* z1, const float* p2,
                                       const uint8_t* c2, const float* z2, int64_t n, int K, const float* weight,
                                       float scale, const float* dloss, float* g1, float* gz1, float* g2, float* gz2,
                                       void* ws, uint32_t flags, cudaStream_t s);
// The GIoU (variant 1) / DIoU (variant 2) terms of the loss (loss_variants.cu).
int64_t loss_var_partials(int64_t n);
dgal_status launch_loss_var_fwd(int variant, const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2,
                                int64_t n, int K, const float* weight, float scale, const float* u, float* ah,
                                uint64_t* aux, float* partials, cudaStream_t s);
dgal_status launch_loss_var_bwd(int variant, const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2,
                                int64_t n, int K, const float* weight, float scale, const float* dloss, const float* u,
                                const float* ah, const uint64_t* aux, float* g1, float* g2,
                                cudaStream_t s);
dgal_status launch_batched(int S, const int64_t* a_off, const int64_t* b_off, const int64_t* out_off,
                           const float* a, const uint8_t* ca, const float* b, const uint8_t* cb, int K, float* iou,
                           uint8_t* nx, void* ws, uint32_t flags, const BatchedConfig& cfg, cudaStream_t s);

} // namespace dgal
