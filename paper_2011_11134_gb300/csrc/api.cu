// C ABI of libdgal (declared in include/dgal.h): argument validation,
// per-thread error messages, the device status word, CUDA-graph capture of
// the ragged batch, and the launch-shape autotuner with its JSON cache.
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "dgal_geom.cuh"
#include "dgal_internal.h"

namespace dgal {

static thread_local std::string t_last_error;

dgal_status fail(dgal_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_last_error = buf;
    return st;
}

dgal_status check_launch(const char* what) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(DGAL_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
    return DGAL_OK;
}

namespace {
std::mutex g_mu;
std::map<int, int> g_sms;
std::map<int, uint32_t*> g_status_ptr;
std::map<std::pair<int, int>, BatchedConfig> g_cfg; // (device, K)

int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d;
}
} // namespace

int sm_count() {
    const int d = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_sms.find(d);
    if (it != g_sms.end()) return it->second;
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d);
    if (n <= 0) n = 1;
    g_sms[d] = n;
    return n;
}

uint32_t* device_status_ptr() {
    const int d = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_status_ptr.find(d);
    if (it != g_status_ptr.end()) return it->second;
    uint32_t* p = status_symbol_address();
    g_status_ptr[d] = p;
    return p;
}

BatchedConfig batched_config(int K) {
    const int d = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cfg.find({d, K});
    if (it != g_cfg.end()) return it->second;
    return BatchedConfig{4096, 128, 4}; // 32 x 128 tiles, four blocks per SM
}

void set_batched_config(int K, BatchedConfig c) {
    const int d = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    g_cfg[{d, K}] = c;
}

namespace {
std::map<std::pair<int, int>, PairedConfig> g_pcfg; // (device, K)
// Untuned default: groups of 8 lanes below 1024 quadrilateral pairs (where
// both shapes are within a few microseconds of the launch floor).
constexpr int64_t kGroupBelowDefault = 1024;
} // namespace

PairedConfig paired_config(int K) {
    const int d = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_pcfg.find({d, K});
    if (it != g_pcfg.end()) return it->second;
    return PairedConfig{K == 4 ? kGroupBelowDefault : 0};
}

void set_paired_config(int K, PairedConfig c) {
    const int d = current_device();
    std::lock_guard<std::mutex> lk(g_mu);
    g_pcfg[{d, K}] = c;
}

} // namespace dgal

using namespace dgal;

namespace {

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

dgal_status check_K(int K) {
    if (K != 4 && K != 8) return fail(DGAL_ERR_UNSUPPORTED_K, "K = %d is not supported (K must be 4 or 8)", K);
    return DGAL_OK;
}

dgal_status check_poly_ptr(const void* p, const char* name) {
    if (!p) return fail(DGAL_ERR_INVALID_ARG, "%s is NULL", name);
    if (!aligned(p, 16)) return fail(DGAL_ERR_ALIGNMENT, "%s is not 16-byte aligned", name);
    return DGAL_OK;
}

#define DGAL_TRY(expr)                  \
    do {                                \
        dgal_status _st = (expr);       \
        if (_st != DGAL_OK) return _st; \
    } while (0)

// DGAL_VALIDATE: the convexity / orientation check of a call's polygon
// arrays, launched before its kernels on the same stream
dgal_status maybe_validate(uint32_t flags, const float* p, const uint8_t* c, int64_t n, int K, cudaStream_t s) {
    if (!(flags & DGAL_VALIDATE)) return DGAL_OK;
    return launch_validate(p, c, n, K, nullptr, s);
}

} // namespace

extern "C" {

int dgal_version(void) { return 100; }

const char* dgal_last_error(void) { return t_last_error.c_str(); }

dgal_status dgal_validate_polygons(const float* p, const uint8_t* c, int64_t n, int K, uint8_t* bad, void* stream) {
    t_last_error.clear();
    DGAL_TRY(check_K(K));
    if (n < 0) return fail(DGAL_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    if (n == 0) return DGAL_OK;
    DGAL_TRY(check_poly_ptr(p, "p"));
    return launch_validate(p, c, n, K, bad, (cudaStream_t)stream);
}

dgal_status dgal_iou_paired(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                            int K, float* iou, uint8_t* nx, uint8_t* xflags, uint8_t* degen, uint32_t flags,
                            void* stream) {
    t_last_error.clear();
    DGAL_TRY(check_K(K));
    if (n < 0) return fail(DGAL_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    if (n == 0) return DGAL_OK;
    DGAL_TRY(check_poly_ptr(p1, "p1"));
    DGAL_TRY(check_poly_ptr(p2, "p2"));
    if (!iou) return fail(DGAL_ERR_INVALID_ARG, "iou is NULL");
    if (!aligned(iou, 4)) return fail(DGAL_ERR_ALIGNMENT, "iou is not 4-byte aligned");
    if ((nx == nullptr) != (xflags == nullptr))
        return fail(DGAL_ERR_INVALID_ARG, "nx and xflags must be both NULL or both set");
    if (xflags && !aligned(xflags, K == 4 ? 8 : 16))
        return fail(DGAL_ERR_ALIGNMENT, "xflags is not %d-byte aligned", K == 4 ? 8 : 16);
    DGAL_TRY(maybe_validate(flags, p1, c1, n, K, (cudaStream_t)stream));
    DGAL_TRY(maybe_validate(flags, p2, c2, n, K, (cudaStream_t)stream));
    return launch_paired_fwd(p1, c1, p2, c2, n, K, iou, nx, xflags, degen, flags, (cudaStream_t)stream);
}

dgal_status dgal_iou_backward(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                              int K, const float* grad_iou, const uint8_t* nx, const uint8_t* xflags,
                              float* grad_p1, float* grad_p2, uint32_t flags, void* stream) {
    t_last_error.clear();
    DGAL_TRY(check_K(K));
    if (n < 0) return fail(DGAL_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    if (n == 0) return DGAL_OK;
    DGAL_TRY(check_poly_ptr(p1, "p1"));
    DGAL_TRY(check_poly_ptr(p2, "p2"));
    DGAL_TRY(check_poly_ptr(grad_p1, "grad_p1"));
    DGAL_TRY(check_poly_ptr(grad_p2, "grad_p2"));
    if (!grad_iou) return fail(DGAL_ERR_INVALID_ARG, "grad_iou is NULL");
    if (!aligned(grad_iou, 4)) return fail(DGAL_ERR_ALIGNMENT, "grad_iou is not 4-byte aligned");
    if ((nx == nullptr) != (xflags == nullptr))
        return fail(DGAL_ERR_INVALID_ARG, "nx and xflags must be both NULL or both set");
    if (xflags && !aligned(xflags, K == 4 ? 8 : 16))
        return fail(DGAL_ERR_ALIGNMENT, "xflags is not %d-byte aligned", K == 4 ? 8 : 16);
    DGAL_TRY(maybe_validate(flags, p1, c1, n, K, (cudaStream_t)stream));
    DGAL_TRY(maybe_validate(flags, p2, c2, n, K, (cudaStream_t)stream));
    return launch_paired_bwd(p1, c1, p2, c2, n, K, grad_iou, nx, xflags, grad_p1, grad_p2, flags,
                             (cudaStream_t)stream);
}

dgal_status dgal_iou_fwd_bwd(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2,
                             const float* grad_iou, int64_t n, int K, float* iou, float* grad_p1, float* grad_p2,
                             uint8_t* nx, uint8_t* xflags, uint32_t flags, void* stream) {
    t_last_error.clear();
    DGAL_TRY(check_K(K));
    if (n < 0) return fail(DGAL_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    if (n == 0) return DGAL_OK;
    DGAL_TRY(check_poly_ptr(p1, "p1"));
    DGAL_TRY(check_poly_ptr(p2, "p2"));
    DGAL_TRY(check_poly_ptr(grad_p1, "grad_p1"));
    DGAL_TRY(check_poly_ptr(grad_p2, "grad_p2"));
    if (!grad_iou || !iou) return fail(DGAL_ERR_INVALID_ARG, "grad_iou or iou is NULL");
    if (!aligned(grad_iou, 4) || !aligned(iou, 4)) return fail(DGAL_ERR_ALIGNMENT, "grad_iou or iou is not 4-byte aligned");
    const cudaStream_t s = (cudaStream_t)stream;
    DGAL_TRY(maybe_validate(flags, p1, c1, n, K, s));
    DGAL_TRY(maybe_validate(flags, p2, c2, n, K, s));
    if (K == 4) return launch_paired_fused(p1, c1, p2, c2, n, K, grad_iou, iou, grad_p1, grad_p2, flags, s);
    // K = 8: the forward saves the flags in the caller's scratch, the backward reads them
    if (!nx || !xflags) return fail(DGAL_ERR_INVALID_ARG, "K = 8 needs nx and xflags scratch");
    if (!aligned(xflags, 16)) return fail(DGAL_ERR_ALIGNMENT, "xflags is not 16-byte aligned");
    const dgal_status r = launch_paired_fwd(p1, c1, p2, c2, n, K, iou, nx, xflags, nullptr, flags, s);
    if (r != DGAL_OK) return r;
    return launch_paired_bwd(p1, c1, p2, c2, n, K, grad_iou, nx, xflags, grad_p1, grad_p2, flags, s);
}

dgal_status dgal_iou_pairwise(const float* a, const uint8_t* ca, int64_t N, const float* b, const uint8_t* cb,
                              int64_t M, int K, float* iou, uint8_t* nx, uint32_t flags, void* stream) {
    t_last_error.clear();
    DGAL_TRY(check_K(K));
    if (N < 0 || M < 0) return fail(DGAL_ERR_INVALID_ARG, "negative size N = %lld, M = %lld", (long long)N, (long long)M);
    if (N == 0 || M == 0) return DGAL_OK;
    if (N > (int64_t)1 << 40 || M > (int64_t)1 << 40) return fail(DGAL_ERR_INVALID_ARG, "N x M too large");
    DGAL_TRY(check_poly_ptr(a, "a"));
    DGAL_TRY(check_poly_ptr(b, "b"));
    if (!iou) return fail(DGAL_ERR_INVALID_ARG, "iou is NULL");
    if (!aligned(iou, 4)) return fail(DGAL_ERR_ALIGNMENT, "iou is not 4-byte aligned");
    DGAL_TRY(maybe_validate(flags, a, ca, N, K, (cudaStream_t)stream));
    DGAL_TRY(maybe_validate(flags, b, cb, M, K, (cudaStream_t)stream));
    return launch_pairwise(a, ca, N, b, cb, M, K, iou, nx, flags, (cudaStream_t)stream);
}

namespace {
dgal_status check_z_ptr(const void* p, const char* name) {
    if (!p) return fail(DGAL_ERR_INVALID_ARG, "%s is NULL", name);
    if (!aligned(p, 8)) return fail(DGAL_ERR_ALIGNMENT, "%s is not 8-byte aligned", name);
    return DGAL_OK;
}
} // namespace

dgal_status dgal_iou3d_paired(const float* p1, const uint8_t* c1, const float* z1, const float* p2, const uint8_t* c2,
                              const float* z2, int64_t n, int K, float* iou, uint8_t* nx, uint8_t* xflags,
                              uint8_t* degen, uint32_t flags, void* stream) {
    t_last_error.clear();
    DGAL_TRY(check_K(K));
    if (n < 0) return fail(DGAL_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    if (n == 0) return DGAL_OK;
    DGAL_TRY(check_poly_ptr(p1, "p1"));
    DGAL_TRY(check_poly_ptr(p2, "p2"));
    DGAL_TRY(check_z_ptr(z1, "z1"));
    DGAL_TRY(check_z_ptr(z2, "z2"));
    if (!iou) return fail(DGAL_ERR_INVALID_ARG, "iou is NULL");
    if (!aligned(iou, 4)) return fail(DGAL_ERR_ALIGNMENT, "iou is not 4-byte aligned");
    if ((nx == nullptr) != (xflags == nullptr))
        return fail(DGAL_ERR_INVALID_ARG, "nx and xflags must be both NULL or both set");
    if (xflags && !aligned(xflags, K == 4 ? 8 : 16))
        return fail(DGAL_ERR_ALIGNMENT, "xflags is not %d-byte aligned", K == 4 ? 8 : 16);
    DGAL_TRY(maybe_validate(flags, p1, c1, n, K, (cudaStream_t)stream));
    DGAL_TRY(maybe_validate(flags, p2, c2, n, K, (cudaStream_t)stream));
    return launch_paired3d_fwd(p1, c1, z1, p2, c2, z2, n, K, iou, nx, xflags, degen, flags, (cudaStream_t)stream);
}

dgal_status dgal_iou3d_backward(const float* p1, const uint8_t* c1, const float* z1, const float* p2,
                                const uint8_t* c2, const float* z2, int64_t n, int K, const float* grad_iou,
                                const uint8_t* nx, const uint8_t* xflags, float* grad_p1, float* grad_z1,
                                float* grad_p2, float* grad_z2, uint32_t flags, void* stream) {
    t_last_error.clear();
    DGAL_TRY(check_K(K));
    if (n < 0) return fail(DGAL_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    if (n == 0) return DGAL_OK;
    DGAL_TRY(check_poly_ptr(p1, "p1"));
    DGAL_TRY(check_poly_ptr(p2, "p2"));
    DGAL_TRY(check_z_ptr(z1, "z1"));
    DGAL_TRY(check_z_ptr(z2, "z2"));
    DGAL_TRY(check_poly_ptr(grad_p1, "grad_p1"));
    DGAL_TRY(check_poly_ptr(grad_p2, "grad_p2"));
    DGAL_TRY(check_z_ptr(grad_z1, "grad_z1"));
    DGAL_TRY(check_z_ptr(grad_z2, "grad_z2"));
    if (!grad_iou) return fail(DGAL_ERR_INVALID_ARG, "grad_iou is NULL");
    if (!aligned(grad_iou, 4)) return fail(DGAL_ERR_ALIGNMENT, "grad_iou is not 4-byte aligned");
    if ((nx == nullptr) != (xflags == nullptr))
        return fail(DGAL_ERR_INVALID_ARG, "nx and xflags must be both NULL or both set");
    if (xflags && !aligned(xflags, K == 4 ? 8 : 16))
        return fail(DGAL_ERR_ALIGNMENT, "xflags is not %d-byte aligned", K == 4 ? 8 : 16);
    DGAL_TRY(maybe_validate(flags, p1, c1, n, K, (cudaStream_t)stream));
    DGAL_TRY(maybe_validate(flags, p2, c2, n, K, (cudaStream_t)stream));
    return launch_paired3d_bwd(p1, c1, z1, p2, c2, z2, n, K, grad_iou, nx, xflags, grad_p1, grad_z1, grad_p2, grad_z2,
                               flags, (cudaStream_t)stream);
}

size_t dgal_iou_loss_workspace_bytes(int64_t n, int K) {
    // beyond 2^40 pairs (64 TB of polygons) the size would overflow; no such input fits in memory
    return (n < 0 || n > (int64_t(1) << 40) || (K != 4 && K != 8)) ? 0 : loss_workspace_bytes(n, K);
}

static dgal_status check_loss_flags(uint32_t flags, bool three_d) {
    const uint32_t var = flags & (DGAL_LOSS_GIOU | DGAL_LOSS_DIOU);
    if (var == (DGAL_LOSS_GIOU | DGAL_LOSS_DIOU))
        return fail(DGAL_ERR_INVALID_ARG, "DGAL_LOSS_GIOU and DGAL_LOSS_DIOU exclude each other");
    if (var && three_d) return fail(DGAL_ERR_INVALID_ARG, "the 3D IoU loss takes neither DGAL_LOSS_GIOU nor DGAL_LOSS_DIOU");
    return DGAL_OK;
}

static dgal_status check_loss_common(const float* p1, const float* p2, int64_t n, int K, const float* weight,
                                     void* workspace, size_t ws_bytes) {
    DGAL_TRY(check_poly_ptr(p1, "p1"));
    DGAL_TRY(check_poly_ptr(p2, "p2"));
    if (weight && !aligned(weight, 4)) return fail(DGAL_ERR_ALIGNMENT, "weight is not 4-byte aligned");
    if (!workspace) return fail(DGAL_ERR_WORKSPACE, "workspace is NULL");
    if (!aligned(workspace, 16)) return fail(DGAL_ERR_ALIGNMENT, "workspace is not 16-byte aligned");
    if (ws_bytes < loss_workspace_bytes(n, K))
        return fail(DGAL_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", ws_bytes, loss_workspace_bytes(n, K));
    return DGAL_OK;
}

dgal_status dgal_iou_loss_backward(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                                   int K, const float* weight, float scale, const float* dloss, float* grad_p1,
                                   float* grad_p2, void* workspace, size_t ws_bytes, uint32_t flags, void* stream) {
    t_last_error.clear();
    if (K != 4 && K != 8) return fail(DGAL_ERR_UNSUPPORTED_K, "K must be 4 or 8 (got %d)", K);
    if (n < 0) return fail(DGAL_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    DGAL_TRY(check_loss_flags(flags, false));
    if (n == 0) return DGAL_OK;
    DGAL_TRY(check_poly_ptr(grad_p1, "grad_p1"));
    DGAL_TRY(check_poly_ptr(grad_p2, "grad_p2"));
    if (dloss && !aligned(dloss, 4)) return fail(DGAL_ERR_ALIGNMENT, "dloss is not 4-byte aligned");
    DGAL_TRY(check_loss_common(p1, p2, n, K, weight, workspace, ws_bytes));
    return launch_iou_loss_backward(p1, c1, p2, c2, n, K, weight, scale, dloss, grad_p1, grad_p2, workspace, flags,
                                    (cudaStream_t)stream);
}

dgal_status dgal_iou3d_loss_backward(const float* p1, const uint8_t* c1, const float* z1, const float* p2,
                                     const uint8_t* c2, const float* z2, int64_t n, int K, const float* weight,
                                     float scale, const float* dloss, float* grad_p1, float* grad_z1, float* grad_p2,
                                     float* grad_z2, void* workspace, size_t ws_bytes, uint32_t flags, void* stream) {
    t_last_error.clear();
    if (K != 4 && K != 8) return fail(DGAL_ERR_UNSUPPORTED_K, "K must be 4 or 8 (got %d)", K);
    if (n < 0) return fail(DGAL_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    DGAL_TRY(check_loss_flags(flags, true));
    if (n == 0) return DGAL_OK;
    DGAL_TRY(check_z_ptr(z1, "z1"));
    DGAL_TRY(check_z_ptr(z2, "z2"));
    DGAL_TRY(check_poly_ptr(grad_p1, "grad_p1"));
    DGAL_TRY(check_poly_ptr(grad_p2, "grad_p2"));
    DGAL_TRY(check_z_ptr(grad_z1, "grad_z1"));
    DGAL_TRY(check_z_ptr(grad_z2, "grad_z2"));
    if (dloss && !aligned(dloss, 4)) return fail(DGAL_ERR_ALIGNMENT, "dloss is not 4-byte aligned");
    DGAL_TRY(check_loss_common(p1, p2, n, K, weight, workspace, ws_bytes));
    return launch_iou3d_loss_backward(p1, c1, z1, p2, c2, z2, n, K, weight, scale, dloss, grad_p1, grad_z1, grad_p2,
                                      grad_z2, workspace, flags, (cudaStream_t)stream);
}

dgal_status dgal_iou_loss(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n, int K,
                          const float* weight, float scale, float* loss, float* iou, float* grad_p1, float* grad_p2,
                          void* workspace, size_t ws_bytes, uint32_t flags, void* stream) {
    t_last_error.clear();
    if (K != 4 && K != 8) return fail(DGAL_ERR_UNSUPPORTED_K, "K must be 4 or 8 (got %d)", K);
    DGAL_TRY(check_loss_flags(flags, false));
    if (n < 0) return fail(DGAL_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    if (!loss) return fail(DGAL_ERR_INVALID_ARG, "loss is NULL");
    if (!aligned(loss, 4)) return fail(DGAL_ERR_ALIGNMENT, "loss is not 4-byte aligned");
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), (cudaStream_t)stream);
        return e == cudaSuccess ? DGAL_OK : fail(DGAL_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    }
    DGAL_TRY(check_poly_ptr(p1, "p1"));
    DGAL_TRY(check_poly_ptr(p2, "p2"));
    if ((grad_p1 == nullptr) != (grad_p2 == nullptr))
        return fail(DGAL_ERR_INVALID_ARG, "grad_p1 and grad_p2 must be both NULL or both set");
    if (grad_p1) {
        DGAL_TRY(check_poly_ptr(grad_p1, "grad_p1"));
        DGAL_TRY(check_poly_ptr(grad_p2, "grad_p2"));
    }
    if (weight && !aligned(weight, 4)) return fail(DGAL_ERR_ALIGNMENT, "weight is not 4-byte aligned");
    if (iou && !aligned(iou, 4)) return fail(DGAL_ERR_ALIGNMENT, "iou is not 4-byte aligned");
    if (!workspace) return fail(DGAL_ERR_WORKSPACE, "workspace is NULL");
    if (!aligned(workspace, 16)) return fail(DGAL_ERR_ALIGNMENT, "workspace is not 16-byte aligned");
    if (ws_bytes < loss_workspace_bytes(n, K))
        return fail(DGAL_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", ws_bytes, loss_workspace_bytes(n, K));
    DGAL_TRY(maybe_validate(flags, p1, c1, n, K, (cudaStream_t)stream));
    DGAL_TRY(maybe_validate(flags, p2, c2, n, K, (cudaStream_t)stream));
    return launch_iou_loss(p1, c1, p2, c2, n, K, weight, scale, loss, iou, grad_p1, grad_p2, workspace, flags,
                           (cudaStream_t)stream);
}

dgal_status dgal_iou3d_loss(const float* p1, const uint8_t* c1, const float* z1, const float* p2, const uint8_t* c2,
                            const float* z2, int64_t n, int K, const float* weight, float scale, float* loss,
                            float* iou, float* grad_p1, float* grad_z1, float* grad_p2, float* grad_z2,
                            void* workspace, size_t ws_bytes, uint32_t flags, void* stream) {
    t_last_error.clear();
    if (K != 4 && K != 8) return fail(DGAL_ERR_UNSUPPORTED_K, "K must be 4 or 8 (got %d)", K);
    DGAL_TRY(check_loss_flags(flags, true));
    if (n < 0) return fail(DGAL_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    if (!loss) return fail(DGAL_ERR_INVALID_ARG, "loss is NULL");
    if (!aligned(loss, 4)) return fail(DGAL_ERR_ALIGNMENT, "loss is not 4-byte aligned");
    if (n == 0) {
        cudaError_t e = cudaMemsetAsync(loss, 0, sizeof(float), (cudaStream_t)stream);
        return e == cudaSuccess ? DGAL_OK : fail(DGAL_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    }
    DGAL_TRY(check_poly_ptr(p1, "p1"));
    DGAL_TRY(check_poly_ptr(p2, "p2"));
    DGAL_TRY(check_z_ptr(z1, "z1"));
    DGAL_TRY(check_z_ptr(z2, "z2"));
    const bool any_g = grad_p1 || grad_p2 || grad_z1 || grad_z2;
    if (any_g && !(grad_p1 && grad_p2 && grad_z1 && grad_z2))
        return fail(DGAL_ERR_INVALID_ARG, "grad_p1, grad_z1, grad_p2, grad_z2 must be all NULL or all set");
    if (any_g) {
        DGAL_TRY(check_poly_ptr(grad_p1, "grad_p1"));
        DGAL_TRY(check_poly_ptr(grad_p2, "grad_p2"));
        DGAL_TRY(check_z_ptr(grad_z1, "grad_z1"));
        DGAL_TRY(check_z_ptr(grad_z2, "grad_z2"));
    }
    if (weight && !aligned(weight, 4)) return fail(DGAL_ERR_ALIGNMENT, "weight is not 4-byte aligned");
    if (iou && !aligned(iou, 4)) return fail(DGAL_ERR_ALIGNMENT, "iou is not 4-byte aligned");
    if (!workspace) return fail(DGAL_ERR_WORKSPACE, "workspace is NULL");
    if (!aligned(workspace, 16)) return fail(DGAL_ERR_ALIGNMENT, "workspace is not 16-byte aligned");
    if (ws_bytes < loss_workspace_bytes(n, K))
        return fail(DGAL_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", ws_bytes, loss_workspace_bytes(n, K));
    DGAL_TRY(maybe_validate(flags, p1, c1, n, K, (cudaStream_t)stream));
    DGAL_TRY(maybe_validate(flags, p2, c2, n, K, (cudaStream_t)stream));
    return launch_iou3d_loss(p1, c1, z1, p2, c2, z2, n, K, weight, scale, loss, iou, grad_p1, grad_z1, grad_p2, grad_z2,
                             workspace, flags, (cudaStream_t)stream);
}

size_t dgal_batched_workspace_bytes(int S, int K) {
    (void)K;
    return S < 0 ? 0 : batched_workspace_bytes(S);
}

} // extern "C"

namespace dgal {
void clear_last_error() { t_last_error.clear(); }

dgal_status check_batched_args(int S, const int64_t* a_off, const int64_t* b_off, const int64_t* out_off,
                               const float* a, const float* b, int K, const float* iou) {
    DGAL_TRY(check_K(K));
    if (S < 0) return fail(DGAL_ERR_INVALID_ARG, "S = %d is negative", S);
    if (!a_off || !b_off || !out_off) return fail(DGAL_ERR_INVALID_ARG, "offset arrays must not be NULL");
    if (!aligned(a_off, 8) || !aligned(b_off, 8) || !aligned(out_off, 8))
        return fail(DGAL_ERR_ALIGNMENT, "offset arrays are not 8-byte aligned");
    DGAL_TRY(check_poly_ptr(a, "a"));
    DGAL_TRY(check_poly_ptr(b, "b"));
    if (!iou) return fail(DGAL_ERR_INVALID_ARG, "iou is NULL");
    if (!aligned(iou, 4)) return fail(DGAL_ERR_ALIGNMENT, "iou is not 4-byte aligned");
    return DGAL_OK;
}
} // namespace dgal

extern "C" {

static dgal_status check_batched(int S, const int64_t* a_off, const int64_t* b_off, const int64_t* out_off,
                                 const float* a, const float* b, int K, float* iou, void* ws, size_t ws_bytes) {
    DGAL_TRY(check_batched_args(S, a_off, b_off, out_off, a, b, K, iou));
    if (!ws) return fail(DGAL_ERR_WORKSPACE, "workspace is NULL");
    if (!aligned(ws, 16)) return fail(DGAL_ERR_ALIGNMENT, "workspace is not 16-byte aligned");
    if (ws_bytes < batched_workspace_bytes(S))
        return fail(DGAL_ERR_WORKSPACE, "workspace has %zu bytes, %zu needed", ws_bytes, batched_workspace_bytes(S));
    return DGAL_OK;
}

dgal_status dgal_iou_pairwise_batched(int S, const int64_t* a_off, const int64_t* b_off, const int64_t* out_off,
                                      const float* a, const uint8_t* ca, const float* b, const uint8_t* cb, int K,
                                      float* iou, uint8_t* nx, void* workspace, size_t ws_bytes, uint32_t flags,
                                      void* stream) {
    t_last_error.clear();
    if (S == 0) return DGAL_OK;
    DGAL_TRY(check_batched(S, a_off, b_off, out_off, a, b, K, iou, workspace, ws_bytes));
    return launch_batched(S, a_off, b_off, out_off, a, ca, b, cb, K, iou, nx, workspace, flags, batched_config(K),
                          (cudaStream_t)stream);
}

dgal_status dgal_iou_pairwise_per_scene(int S, const int64_t* a_off_h, const int64_t* b_off_h,
                                        const int64_t* out_off_h, const float* a, const uint8_t* ca, const float* b,
                                        const uint8_t* cb, int K, float* iou, uint8_t* nx, uint32_t flags,
                                        void* stream) {
    t_last_error.clear();
    DGAL_TRY(check_K(K));
    if (S < 0) return fail(DGAL_ERR_INVALID_ARG, "S = %d is negative", S);
    if (S == 0) return DGAL_OK;
    if (!a_off_h || !b_off_h || !out_off_h) return fail(DGAL_ERR_INVALID_ARG, "offset arrays must not be NULL");
    DGAL_TRY(check_poly_ptr(a, "a"));
    DGAL_TRY(check_poly_ptr(b, "b"));
    if (!iou) return fail(DGAL_ERR_INVALID_ARG, "iou is NULL");
    for (int s = 0; s < S; ++s) {
        const int64_t N = a_off_h[s + 1] - a_off_h[s], M = b_off_h[s + 1] - b_off_h[s];
        if (N < 0 || M < 0 || out_off_h[s + 1] - out_off_h[s] != N * M)
            return fail(DGAL_ERR_INVALID_ARG, "scene %d: inconsistent offsets", s);
    }
    for (int s = 0; s < S; ++s) {
        const int64_t N = a_off_h[s + 1] - a_off_h[s], M = b_off_h[s + 1] - b_off_h[s];
        if (N == 0 || M == 0) continue;
        DGAL_TRY(launch_pairwise(a + a_off_h[s] * 2 * K, ca ? ca + a_off_h[s] : nullptr, N, b + b_off_h[s] * 2 * K,
                                 cb ? cb + b_off_h[s] : nullptr, M, K, iou + out_off_h[s],
                                 nx ? nx + out_off_h[s] : nullptr, flags, (cudaStream_t)stream));
    }
    return DGAL_OK;
}

struct dgal_graph_s {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

dgal_status dgal_batched_graph_create(dgal_graph* out, int S, const int64_t* a_off, const int64_t* b_off,
                                      const int64_t* out_off, const float* a, const uint8_t* ca, const float* b,
                                      const uint8_t* cb, int K, float* iou, uint8_t* nx, void* workspace,
                                      size_t ws_bytes, uint32_t flags) {
    t_last_error.clear();
    if (!out) return fail(DGAL_ERR_INVALID_ARG, "graph is NULL");
    *out = nullptr;
    if (S <= 0) return fail(DGAL_ERR_INVALID_ARG, "S = %d: nothing to capture", S);
    DGAL_TRY(check_batched(S, a_off, b_off, out_off, a, b, K, iou, workspace, ws_bytes));
    // resolve cached per-device state before the capture starts
    (void)sm_count();
    (void)device_status_ptr();
    const BatchedConfig cfg = batched_config(K);
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
        return fail(DGAL_ERR_CUDA, "cudaStreamCreate failed");
    dgal_graph_s* g = new dgal_graph_s();
    dgal_status st = DGAL_OK;
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        st = fail(DGAL_ERR_CUDA, "cudaStreamBeginCapture failed");
    } else {
        st = launch_batched(S, a_off, b_off, out_off, a, ca, b, cb, K, iou, nx, workspace, flags, cfg, s);
        cudaError_t e = cudaStreamEndCapture(s, &g->graph);
        if (st == DGAL_OK && e != cudaSuccess) st = fail(DGAL_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
        if (st == DGAL_OK) {
            e = cudaGraphInstantiate(&g->exec, g->graph, 0);
            if (e != cudaSuccess) st = fail(DGAL_ERR_CUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(e));
        }
    }
    cudaStreamDestroy(s);
    if (st != DGAL_OK) {
        if (g->exec) cudaGraphExecDestroy(g->exec);
        if (g->graph) cudaGraphDestroy(g->graph);
        delete g;
        return st;
    }
    *out = g;
    return DGAL_OK;
}

dgal_status dgal_graph_launch(dgal_graph graph, void* stream) {
    t_last_error.clear();
    if (!graph || !graph->exec) return fail(DGAL_ERR_INVALID_ARG, "graph is NULL");
    cudaError_t e = cudaGraphLaunch(graph->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(DGAL_ERR_CUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
    return DGAL_OK;
}

dgal_status dgal_graph_destroy(dgal_graph graph) {
    t_last_error.clear();
    if (!graph) return DGAL_OK;
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
    delete graph;
    return DGAL_OK;
}

dgal_status dgal_get_device_status(uint32_t* out, int clear) {
    t_last_error.clear();
    if (!out) return fail(DGAL_ERR_INVALID_ARG, "out is NULL");
    uint32_t* p = device_status_ptr();
    if (!p) return fail(DGAL_ERR_CUDA, "status word not available on this device");
    cudaError_t e = cudaMemcpy(out, p, sizeof(uint32_t), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(DGAL_ERR_CUDA, "reading status: %s", cudaGetErrorString(e));
    if (clear) {
        e = cudaMemset(p, 0, sizeof(uint32_t));
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return fail(DGAL_ERR_CUDA, "clearing status: %s", cudaGetErrorString(e));
    }
    return DGAL_OK;
}

dgal_status dgal_get_batched_config(int K, int32_t out[3]) {
    t_last_error.clear();
    DGAL_TRY(check_K(K));
    if (!out) return fail(DGAL_ERR_INVALID_ARG, "out is NULL");
    BatchedConfig c = batched_config(K);
    out[0] = c.tile;
    out[1] = c.threads;
    out[2] = c.blocks_sm;
    return DGAL_OK;
}

dgal_status dgal_get_paired_config(int K, int64_t* group_below) {
    t_last_error.clear();
    DGAL_TRY(check_K(K));
    if (!group_below) return fail(DGAL_ERR_INVALID_ARG, "group_below is NULL");
    *group_below = paired_config(K).group_below;
    return DGAL_OK;
}

} // extern "C"

// ---------------------------------------------------------------- autotuner

namespace dgal_tune {

// splitmix64: counter-based generator for the tuner's synthetic boxes
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}
__device__ __forceinline__ float unit(uint64_t z) { return (float)(mix64(z) >> 40) * (1.0f / 16777216.0f); }

// Car-like boxes in a 70 m plane, 40 clusters per scene (the tuning problem).
__global__ void k_synth_boxes(float* __restrict__ out, const int64_t* __restrict__ scene_of_off, int S,
                              int64_t n, uint64_t seed, int K) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int lo = 0, hi = S;
    while (hi - lo > 1) {
        int mid = (lo + hi) >> 1;
        if (scene_of_off[mid] <= k) lo = mid; else hi = mid;
    }
    const uint64_t base = seed * 0x100000001B3ull + (uint64_t)k * 16u;
    const int cl = (int)(unit(base) * 40.f);
    const uint64_t cbase = seed * 7919u + (uint64_t)lo * 131u + (uint64_t)cl;
    const float cx = 70.f * unit(cbase * 3u + 1u), cy = 70.f * unit(cbase * 3u + 2u);
    const float gx = (unit(base + 1) + unit(base + 2) + unit(base + 3) - 1.5f) * 6.f;
    const float gy = (unit(base + 4) + unit(base + 5) + unit(base + 6) - 1.5f) * 6.f;
    const float w = 1.5f + 0.7f * unit(base + 7), l = 3.5f + 1.5f * unit(base + 8);
    const float th = 6.2831853f * unit(base + 9) - 3.1415927f;
    float s, c;
    sincosf(th, &s, &c);
    const float lx[4] = {-l / 2, l / 2, l / 2, -l / 2}, ly[4] = {-w / 2, -w / 2, w / 2, w / 2};
    float* p = out + k * 2 * K;
    for (int v = 0; v < K; ++v) {
        const int q = (K == 4) ? v : (v < 4 ? v : 0);
        p[2 * v] = cx + gx + c * lx[q] - s * ly[q];
        p[2 * v + 1] = cy + gy + s * lx[q] + c * ly[q];
    }
}

std::string device_key(int K) {
    cudaDeviceProp prop;
    int d = 0;
    cudaGetDevice(&d);
    cudaGetDeviceProperties(&prop, d);
    char buf[320];
    snprintf(buf, sizeof(buf), "%s|sm%d%d|K=%d", prop.name, prop.major, prop.minor, K);
    return buf;
}

// A launch shape the ragged-batch kernel accepts: whole warps, at most 256
// threads (the tile's queue codes hold the column in 8 bits), 1 to 64
// resident blocks per SM, a positive tile.  Cache entries outside this are
// ignored.
bool valid_config(int t, int th, int b) {
    return t > 0 && th >= 32 && th <= 256 && th % 32 == 0 && b >= 1 && b <= 64;
}

// Tiny JSON map {"key": [a, b, c], ...} (one line per entry): for a ragged
// batch key [tile, threads, blocks_sm], for a paired key ("...|paired")
// [group_below, 0, 0].
struct Triple {
    long long a, b, c;
};
std::map<std::string, Triple> read_cache(const std::string& path) {
    std::map<std::string, Triple> m;
    FILE* f = fopen(path.c_str(), "r");
    if (!f) return m;
    char line[1024];
    while (fgets(line, sizeof(line), f)) {
        char* q1 = strchr(line, '"');
        if (!q1) continue;
        char* q2 = strchr(q1 + 1, '"');
        if (!q2) continue;
        std::string key(q1 + 1, q2);
        long long t = 0, th = 0, b = 0;
        char* br = strchr(q2, '[');
        if (br && sscanf(br, "[%lld, %lld, %lld]", &t, &th, &b) == 3) m[key] = Triple{t, th, b};
    }
    fclose(f);
    return m;
}

bool write_cache(const std::string& path, const std::map<std::string, Triple>& m) {
    std::string tmp = path + ".tmp";
    FILE* f = fopen(tmp.c_str(), "w");
    if (!f) return false;
    fprintf(f, "{\n");
    size_t k = 0;
    for (auto& kv : m) {
        fprintf(f, "  \"%s\": [%lld, %lld, %lld]%s\n", kv.first.c_str(), kv.second.a, kv.second.b, kv.second.c,
                (++k < m.size()) ? "," : "");
    }
    fprintf(f, "}\n");
    fclose(f);
    return rename(tmp.c_str(), path.c_str()) == 0;
}

// IoU-loss-like quadrilateral pairs for the paired tuning: box a with center
// in [0, 10]^2, sides in [0.5, 4], any angle; box b = a moved by about
// N(0, 0.5) per axis, sides scaled in [0.8, 1.2], turned by up to 0.3.
__global__ void k_synth_pairs(float* __restrict__ p1, float* __restrict__ p2, int64_t n, uint64_t seed) {
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const uint64_t b = seed * 0x9E3779B97F4A7C15ull + (uint64_t)k * 32u;
    const float cx = 10.f * unit(b), cy = 10.f * unit(b + 1);
    const float w = 0.5f + 3.5f * unit(b + 2), h = 0.5f + 3.5f * unit(b + 3);
    const float th = 6.2831853f * unit(b + 4) - 3.1415927f;
    const float dx = (unit(b + 5) + unit(b + 6) + unit(b + 7) - 1.5f), dy = (unit(b + 8) + unit(b + 9) + unit(b + 10) - 1.5f);
    const float w2 = w * (0.8f + 0.4f * unit(b + 11)), h2 = h * (0.8f + 0.4f * unit(b + 12));
    const float th2 = th + 0.6f * unit(b + 13) - 0.3f;
    const float lx[4] = {-0.5f, 0.5f, 0.5f, -0.5f}, ly[4] = {-0.5f, -0.5f, 0.5f, 0.5f};
    float s, c, s2, c2;
    sincosf(th, &s, &c);
    sincosf(th2, &s2, &c2);
    for (int v = 0; v < 4; ++v) {
        p1[k * 8 + 2 * v] = cx + c * w * lx[v] - s * h * ly[v];
        p1[k * 8 + 2 * v + 1] = cy + s * w * lx[v] + c * h * ly[v];
        p2[k * 8 + 2 * v] = cx + dx + c2 * w2 * lx[v] - s2 * h2 * ly[v];
        p2[k * 8 + 2 * v + 1] = cy + dy + s2 * w2 * lx[v] + c2 * h2 * ly[v];
    }
}

} // namespace dgal_tune

using namespace dgal_tune;

// Paired launch shape (config_class 1): for quadrilaterals, the batch size
// below which groups of 8 lanes beat one lane per pair, from timing both
// shapes on the forward + backward of synthetic pairs at sizes 2^10 .. 2^18.
static dgal_status tune_paired(int K, const std::string& path) {
    const std::string key = device_key(K) + "|paired";
    if (!path.empty()) {
        auto m = read_cache(path);
        auto it = m.find(key);
        if (it != m.end() && it->second.a >= 0) {
            set_paired_config(K, PairedConfig{(int64_t)it->second.a});
            return DGAL_OK;
        }
    }
    if (K != 4) { // K = 8 pairs always take groups of 8 lanes
        set_paired_config(K, PairedConfig{0});
        return DGAL_OK;
    }
    const int64_t nmax = 1 << 18;
    float *p1 = nullptr, *p2 = nullptr, *iou = nullptr, *grad = nullptr, *g1 = nullptr, *g2 = nullptr;
    uint8_t *nx = nullptr, *xf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&]() {
        cudaFree(p1); cudaFree(p2); cudaFree(iou); cudaFree(grad); cudaFree(g1); cudaFree(g2); cudaFree(nx); cudaFree(xf);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMalloc(&p1, nmax * 32) != cudaSuccess || cudaMalloc(&p2, nmax * 32) != cudaSuccess ||
        cudaMalloc(&iou, nmax * 4) != cudaSuccess || cudaMalloc(&grad, nmax * 4) != cudaSuccess ||
        cudaMalloc(&g1, nmax * 32) != cudaSuccess || cudaMalloc(&g2, nmax * 32) != cudaSuccess ||
        cudaMalloc(&nx, nmax) != cudaSuccess || cudaMalloc(&xf, nmax * 8) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        return fail(DGAL_ERR_CUDA, "autotune: allocation failed");
    }
    k_synth_pairs<<<(unsigned)(nmax / 256), 256>>>(p1, p2, nmax, 3);
    cudaMemset(grad, 0, nmax * 4);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cleanup();
        return fail(DGAL_ERR_CUDA, "autotune: synthetic input generation failed");
    }
    // time one shape (forced by the threshold) at n pairs: best of 5 steps after one
    auto step_ms = [&](int64_t n, int64_t below) -> float {
        set_paired_config(4, PairedConfig{below});
        float best = 1e30f;
        for (int rep = 0; rep < 6; ++rep) {
            cudaEventRecord(e0, 0);
            launch_paired_fwd(p1, nullptr, p2, nullptr, n, 4, iou, nx, xf, nullptr, kFlagRefine, 0);
            launch_paired_bwd(p1, nullptr, p2, nullptr, n, 4, grad, nx, xf, g1, g2, kFlagRefine, 0);
            cudaEventRecord(e1, 0);
            cudaEventSynchronize(e1);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;
        }
        return best;
    };
    int64_t below = 2 * nmax; // groups everywhere unless one lane per pair wins
    for (int64_t n = 1 << 10; n <= nmax; n <<= 2) {
        const float tg = step_ms(n, INT64_MAX), t1 = step_ms(n, 0);
        if (t1 <= tg) {
            below = n;
            break;
        }
    }
    const cudaError_t e = cudaGetLastError();
    cleanup();
    if (e != cudaSuccess) return fail(DGAL_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
    set_paired_config(4, PairedConfig{below});
    if (!path.empty()) {
        auto m = read_cache(path);
        m[key] = Triple{(long long)below, 0, 0};
        if (!write_cache(path, m)) return fail(DGAL_ERR_INVALID_ARG, "autotune: cannot write %s", path.c_str());
    }
    return DGAL_OK;
}

extern "C" dgal_status dgal_autotune(int K, int config_class, const char* cache_path) {
    t_last_error.clear();
    DGAL_TRY(check_K(K));
    if (config_class != 0 && config_class != 1)
        return fail(DGAL_ERR_INVALID_ARG, "config_class must be 0 (ragged batch) or 1 (paired), got %d", config_class);
    std::string path;
    if (cache_path) path = cache_path;
    else if (const char* env = getenv("DGAL_TUNE_CACHE")) path = env;
    if (config_class == 1) return tune_paired(K, path);
    const std::string key = device_key(K);
    if (!path.empty()) {
        auto m = read_cache(path);
        auto it = m.find(key);
        if (it != m.end() && valid_config((int)it->second.a, (int)it->second.b, (int)it->second.c)) {
            set_batched_config(K, BatchedConfig{(int)it->second.a, (int)it->second.b, (int)it->second.c});
            return DGAL_OK;
        }
    }

    // synthetic ragged problem: 64 scenes, N_s in [50, 3000], M_s in [5, 200]
    const int S = 64;
    std::vector<int64_t> ao(S + 1, 0), bo(S + 1, 0), oo(S + 1, 0);
    uint64_t lcg = 0x2545F4914F6CDD1Dull;
    auto nextu = [&lcg](uint64_t m) {
        lcg = lcg * 6364136223846793005ull + 1442695040888963407ull;
        return (lcg >> 33) % m;
    };
    for (int s = 0; s < S; ++s) {
        const int64_t N = 50 + (int64_t)nextu(2951), M = 5 + (int64_t)nextu(196);
        ao[s + 1] = ao[s] + N;
        bo[s + 1] = bo[s] + M;
        oo[s + 1] = oo[s] + N * M;
    }
    const size_t ws_bytes = batched_workspace_bytes(S);
    float *a = nullptr, *b = nullptr, *iou = nullptr;
    uint8_t* nx = nullptr;
    int64_t* offs = nullptr;
    void* ws = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    dgal_status st = DGAL_OK;
    auto cleanup = [&]() {
        cudaFree(a); cudaFree(b); cudaFree(iou); cudaFree(nx); cudaFree(offs); cudaFree(ws);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    if (cudaMalloc(&a, ao[S] * 2 * K * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&b, bo[S] * 2 * K * sizeof(float)) != cudaSuccess ||
        cudaMalloc(&iou, oo[S] * sizeof(float)) != cudaSuccess || cudaMalloc(&nx, oo[S]) != cudaSuccess ||
        cudaMalloc(&offs, 3 * (S + 1) * sizeof(int64_t)) != cudaSuccess || cudaMalloc(&ws, ws_bytes) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cleanup();
        return fail(DGAL_ERR_CUDA, "autotune: allocation failed");
    }
    cudaMemcpy(offs, ao.data(), (S + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    cudaMemcpy(offs + (S + 1), bo.data(), (S + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    cudaMemcpy(offs + 2 * (S + 1), oo.data(), (S + 1) * sizeof(int64_t), cudaMemcpyHostToDevice);
    k_synth_boxes<<<(unsigned)((ao[S] + 255) / 256), 256>>>(a, offs, S, ao[S], 1, K);
    k_synth_boxes<<<(unsigned)((bo[S] + 255) / 256), 256>>>(b, offs + (S + 1), S, bo[S], 2, K);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cleanup();
        return fail(DGAL_ERR_CUDA, "autotune: synthetic input generation failed");
    }
    const int tiles[] = {1024, 2048, 4096}; // entries per tile: rows x threads
    const int threads[] = {128, 256};
    const int bps[] = {2, 4, 8, 12};
    BatchedConfig best{1024, 128, 8};
    float best_ms = 1e30f;
    for (int t : tiles)
        for (int th : threads)
            for (int bp : bps) {
                if (th * bp > 2048) continue;
                BatchedConfig c{t, th, bp};
                float ms_min = 1e30f;
                for (int rep = 0; rep < 4 && st == DGAL_OK; ++rep) {
                    cudaEventRecord(e0, 0);
                    st = launch_batched(S, offs, offs + (S + 1), offs + 2 * (S + 1), a, nullptr, b, nullptr, K, iou,
                                        nx, ws, kFlagRefine, c, 0);
                    cudaEventRecord(e1, 0);
                    cudaEventSynchronize(e1);
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    if (rep > 0 && ms < ms_min) ms_min = ms;
                }
                if (st != DGAL_OK) {
                    cleanup();
                    return st;
                }
                if (ms_min < best_ms) {
                    best_ms = ms_min;
                    best = c;
                }
            }
    cleanup();
    set_batched_config(K, best);
    if (!path.empty()) {
        auto m = read_cache(path);
        m[key] = Triple{best.tile, best.threads, best.blocks_sm};
        if (!write_cache(path, m)) return fail(DGAL_ERR_INVALID_ARG, "autotune: cannot write %s", path.c_str());
    }
    return DGAL_OK;
}
