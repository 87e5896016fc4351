// Paired 3D IoU: the paired kernels in 3D mode (bird's-eye-view polygon
// intersection times the overlap of the vertical extents, paper Sec. IV-A).
//
// Forward (paper Sec. II-B `iou`): loads both polygons with 128-bit loads,
// clips in registers (dgal_geom.cuh), stores IoU (4 B), nx (1 B) and the
// 2K code bytes as one 64/128-bit store, plus an optional degeneracy byte.
// Backward (paper Sec. II-B `iou_backward`): reads the polygons, dL/dIoU and
// the recorded (nx, xflags), or recomputes the clip, and writes both
// gradients with 128-bit stores.
#include "paired_launch.cuh"

namespace dgal {

dgal_status launch_paired3d_fwd(const float* p1, const uint8_t* c1, const float* z1, const float* p2,
                                const uint8_t* c2, const float* z2, int64_t n, int K, float* iou, uint8_t* nx,
                                uint8_t* xflags, uint8_t* degen, uint32_t flags, cudaStream_t s) {
    if (!device_status_ptr()) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    fwd_any<false, true>(p1, c1, p2, c2, n, K, iou, nx, xflags, degen, flags, s, LossArgs{nullptr, 0.f, nullptr},
                         ZArgs{z1, z2, nullptr, nullptr});
    return check_launch("paired 3D forward");
}

dgal_status launch_paired3d_bwd(const float* p1, const uint8_t* c1, const float* z1, const float* p2,
                                const uint8_t* c2, const float* z2, int64_t n, int K, const float* grad,
                                const uint8_t* nx, const uint8_t* xflags, float* g1, float* gz1, float* g2, float* gz2,
                                uint32_t flags, cudaStream_t s) {
    if (!device_status_ptr()) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    bwd_any<false, true>(p1, c1, p2, c2, n, K, grad, nx, xflags, g1, g2, flags, s, LossArgs{nullptr, 0.f, nullptr},
                         ZArgs{z1, z2, gz1, gz2});
    return check_launch("paired 3D backward");
}

dgal_status launch_iou3d_loss(const float* p1, const uint8_t* c1, const float* z1, const float* p2, const uint8_t* c2,
                              const float* z2, int64_t n, int K, const float* weight, float scale, float* loss,
                              float* iou, float* g1, float* gz1, float* g2, float* gz2, void* ws, uint32_t flags,
                              cudaStream_t s) {
    if (!device_status_ptr()) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    return iou_loss_passes<true>(p1, c1, p2, c2, n, K, weight, scale, loss, iou, g1, g2, ZArgs{z1, z2, gz1, gz2}, ws,
                                 flags, s);
}

dgal_status launch_iou3d_loss_backward(const float* p1, const uint8_t* c1, const float* z1, const float* p2,
                                       const uint8_t* c2, const float* z2, int64_t n, int K, const float* weight,
                                       float scale, const float* dloss, float* g1, float* gz1, float* g2, float* gz2,
                                       void* ws, uint32_t flags, cudaStream_t s) {
    if (!device_status_ptr()) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    return iou_loss_backward<true>(p1, c1, p2, c2, n, K, weight, scale, dloss, nullptr, g1, g2,
                                   ZArgs{z1, z2, gz1, gz2}, ws, flags, s);
}

} // namespace dgal
