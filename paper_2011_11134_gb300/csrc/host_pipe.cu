// Paired IoU forward + backward on host-resident data.
//
// The paired kernels take a few tens of microseconds per million pairs; for
// data that lives in host memory the host link dominates.  Two forms:
//
// Direct (K = 4, every buffer pinned and mapped into the device's address
// space): one kernel reads the polygons (and counts) and dL/dIoU from host
// memory and writes IoU and both gradients back, the clip state staying in
// registers between the forward and the backward (k_paired_fused).  Loads
// from both directions are in flight together, and nothing is staged.  (A
// K = 8 one-pass kernel measured slower than the staged form: it needs 168
// registers, and its warp path reads the polygons again over the link.)
//
// Staged (otherwise): the pairs go in chunks; for chunk c in staging slot
// c mod 3 (the counts, when given, travel with the polygons):
//   copy-in stream   host -> slot: p1, p2, dL/dIoU         (event in[s])
//   caller's stream  paired forward (flags kept in the slot) and backward
//                    from those flags                       (event done[s])
//   copy-out stream  slot -> host: IoU, dL/dp1, dL/dp2      (event out[s])
// so the copies in both directions overlap each other and the kernels.  A
// slot's inputs are rewritten only after its previous kernels finished, and
// its outputs only after they were copied out.  The copy streams first wait
// for the work already on the caller's stream, and the caller's stream
// finally waits for the last copies, so the call is ordered on the caller's
// stream like any other.  Streams and events are created once per device
// (the first call on a device) and reused; device memory is the caller's
// workspace.
#include <map>
#include <mutex>

#include "dgal_internal.h"

namespace dgal {
namespace {

constexpr int kSlots = 3;

struct PipeState {
    cudaStream_t in = nullptr, out = nullptr;
    cudaEvent_t entry = nullptr;
    cudaEvent_t ev_in[kSlots], ev_done[kSlots], ev_out[kSlots];
};

std::mutex g_pipe_mu;
std::map<int, PipeState> g_pipe; // device ordinal -> streams and events

dgal_status pipe_state(PipeState** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(DGAL_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(g_pipe_mu);
    auto it = g_pipe.find(dev);
    if (it != g_pipe.end()) {
        *out = &it->second;
        return DGAL_OK;
    }
    PipeState st;
    e = cudaStreamCreateWithFlags(&st.in, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st.out, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st.entry, cudaEventDisableTiming);
    for (int s = 0; s < kSlots && e == cudaSuccess; ++s) {
        e = cudaEventCreateWithFlags(&st.ev_in[s], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st.ev_done[s], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&st.ev_out[s], cudaEventDisableTiming);
    }
    if (e != cudaSuccess) return fail(DGAL_ERR_CUDA, "creating the copy streams: %s", cudaGetErrorString(e));
    auto res = g_pipe.emplace(dev, st);
    *out = &res.first->second;
    return DGAL_OK;
}

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

// One slot: p1 | p2 | grad | iou | nx | xflags | g1 | g2 | c1 | c2, each
// 256-byte aligned.
struct SlotLayout {
    size_t p1, p2, grad, iou, nx, xflags, g1, g2, c1, c2, bytes;
};

SlotLayout slot_layout(int64_t chunk, int K) {
    SlotLayout L;
    const size_t poly = (size_t)chunk * K * 2 * sizeof(float);
    size_t o = 0;
    L.p1 = o;
    o += up256(poly);
    L.p2 = o;
    o += up256(poly);
    L.grad = o;
    o += up256((size_t)chunk * 4);
    L.iou = o;
    o += up256((size_t)chunk * 4);
    L.nx = o;
    o += up256((size_t)chunk);
    L.xflags = o;
    o += up256((size_t)chunk * 2 * K);
    L.g1 = o;
    o += up256(poly);
    L.g2 = o;
    o += up256(poly);
    L.c1 = o;
    o += up256((size_t)chunk);
    L.c2 = o;
    o += up256((size_t)chunk);
    L.bytes = o;
    return L;
}

#define PIPE_CUDA(expr)                                                                              \
    do {                                                                                             \
        cudaError_t _e = (expr);                                                                     \
        if (_e != cudaSuccess) return fail(DGAL_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(_e)); \
    } while (0)

// Device address of a host buffer the device can load and store directly
// (pinned and mapped), else NULL.
void* mapped(const void* h) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, h) != cudaSuccess) {
        cudaGetLastError(); // not a CUDA pointer: clear the error
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

} // namespace
} // namespace dgal

using namespace dgal;

extern "C" size_t dgal_iou_host_workspace_bytes(int64_t chunk, int K) {
    // beyond 2^40 pairs per chunk the size would overflow; no such slot fits in memory
    if ((K != 4 && K != 8) || chunk <= 0 || chunk > (int64_t(1) << 40)) return 0;
    return kSlots * slot_layout(chunk, K).bytes;
}

extern "C" dgal_status dgal_iou_fwd_bwd_host(const float* h_p1, const uint8_t* h_c1, const float* h_p2,
                                             const uint8_t* h_c2, const float* h_grad, int64_t n, int K, float* h_iou,
                                             float* h_g1, float* h_g2, void* workspace, size_t ws_bytes, int64_t chunk,
                                             uint32_t flags, void* stream) {
    if (K != 4 && K != 8) return fail(DGAL_ERR_UNSUPPORTED_K, "K = %d is not supported (K must be 4 or 8)", K);
    if (n < 0) return fail(DGAL_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    if (n == 0) return DGAL_OK;
    if (chunk <= 0) return fail(DGAL_ERR_INVALID_ARG, "chunk = %lld must be positive", (long long)chunk);
    if (!h_p1 || !h_p2 || !h_grad || !h_iou || !h_g1 || !h_g2)
        return fail(DGAL_ERR_INVALID_ARG, "a host buffer is NULL");
    if (K == 4) {
        void* d_p1 = mapped(h_p1);
        void* d_p2 = mapped(h_p2);
        void* d_grad = mapped(h_grad);
        void* d_iou = mapped(h_iou);
        void* d_g1 = mapped(h_g1);
        void* d_g2 = mapped(h_g2);
        void* d_c1 = h_c1 ? mapped(h_c1) : nullptr;
        void* d_c2 = h_c2 ? mapped(h_c2) : nullptr;
        // 16-byte vertex loads and stores
        const bool aligned = ((reinterpret_cast<uintptr_t>(d_p1) | reinterpret_cast<uintptr_t>(d_p2) |
                               reinterpret_cast<uintptr_t>(d_g1) | reinterpret_cast<uintptr_t>(d_g2)) & 15u) == 0;
        const bool counts_ok = (!h_c1 || d_c1) && (!h_c2 || d_c2);
        if (d_p1 && d_p2 && d_grad && d_iou && d_g1 && d_g2 && counts_ok && aligned)
            return launch_paired_fused(static_cast<const float*>(d_p1), static_cast<const uint8_t*>(d_c1),
                                       static_cast<const float*>(d_p2), static_cast<const uint8_t*>(d_c2), n, K,
                                       static_cast<const float*>(d_grad), static_cast<float*>(d_iou),
                                       static_cast<float*>(d_g1), static_cast<float*>(d_g2), flags,
                                       (cudaStream_t)stream);
    }
    if (chunk > n) chunk = n; // a slot never needs more than the pairs there are
    if (!workspace) return fail(DGAL_ERR_WORKSPACE, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(workspace) & 255u)
        return fail(DGAL_ERR_ALIGNMENT, "workspace is not 256-byte aligned");
    const SlotLayout L = slot_layout(chunk, K);
    if (ws_bytes < kSlots * L.bytes)
        return fail(DGAL_ERR_WORKSPACE, "workspace of %zu bytes is smaller than the %zu bytes needed", ws_bytes,
                    kSlots * L.bytes);
    PipeState* P = nullptr;
    dgal_status st = pipe_state(&P);
    if (st != DGAL_OK) return st;
    cudaStream_t cs = (cudaStream_t)stream;
    // the copy streams start after the work already queued on the caller's stream
    PIPE_CUDA(cudaEventRecord(P->entry, cs));
    PIPE_CUDA(cudaStreamWaitEvent(P->in, P->entry, 0));
    PIPE_CUDA(cudaStreamWaitEvent(P->out, P->entry, 0));
    const int64_t nchunks = (n + chunk - 1) / chunk;
    const size_t pp = (size_t)K * 2 * sizeof(float); // bytes of one polygon
    for (int64_t c = 0; c < nchunks; ++c) {
        const int s = (int)(c % kSlots);
        const int64_t k0 = c * chunk;
        const int64_t m = (n - k0 < chunk) ? n - k0 : chunk;
        char* base = static_cast<char*>(workspace) + (size_t)s * L.bytes;
        float* d_p1 = reinterpret_cast<float*>(base + L.p1);
        float* d_p2 = reinterpret_cast<float*>(base + L.p2);
        float* d_grad = reinterpret_cast<float*>(base + L.grad);
        float* d_iou = reinterpret_cast<float*>(base + L.iou);
        uint8_t* d_nx = reinterpret_cast<uint8_t*>(base + L.nx);
        uint8_t* d_xf = reinterpret_cast<uint8_t*>(base + L.xflags);
        float* d_g1 = reinterpret_cast<float*>(base + L.g1);
        float* d_g2 = reinterpret_cast<float*>(base + L.g2);
        uint8_t* d_c1 = h_c1 ? reinterpret_cast<uint8_t*>(base + L.c1) : nullptr;
        uint8_t* d_c2 = h_c2 ? reinterpret_cast<uint8_t*>(base + L.c2) : nullptr;
        // inputs: the slot's previous kernels must be done with them
        if (c >= kSlots) PIPE_CUDA(cudaStreamWaitEvent(P->in, P->ev_done[s], 0));
        PIPE_CUDA(cudaMemcpyAsync(d_p1, h_p1 + (size_t)k0 * K * 2, (size_t)m * pp, cudaMemcpyHostToDevice, P->in));
        PIPE_CUDA(cudaMemcpyAsync(d_p2, h_p2 + (size_t)k0 * K * 2, (size_t)m * pp, cudaMemcpyHostToDevice, P->in));
        PIPE_CUDA(cudaMemcpyAsync(d_grad, h_grad + k0, (size_t)m * 4, cudaMemcpyHostToDevice, P->in));
        if (h_c1) PIPE_CUDA(cudaMemcpyAsync(d_c1, h_c1 + k0, (size_t)m, cudaMemcpyHostToDevice, P->in));
        if (h_c2) PIPE_CUDA(cudaMemcpyAsync(d_c2, h_c2 + k0, (size_t)m, cudaMemcpyHostToDevice, P->in));
        PIPE_CUDA(cudaEventRecord(P->ev_in[s], P->in));
        // kernels: inputs arrived, and the slot's previous outputs were copied out
        PIPE_CUDA(cudaStreamWaitEvent(cs, P->ev_in[s], 0));
        if (c >= kSlots) PIPE_CUDA(cudaStreamWaitEvent(cs, P->ev_out[s], 0));
        st = launch_paired_fwd(d_p1, d_c1, d_p2, d_c2, m, K, d_iou, d_nx, d_xf, nullptr, flags, cs, n);
        if (st != DGAL_OK) return st;
        st = launch_paired_bwd(d_p1, d_c1, d_p2, d_c2, m, K, d_grad, d_nx, d_xf, d_g1, d_g2, flags, cs, n);
        if (st != DGAL_OK) return st;
        PIPE_CUDA(cudaEventRecord(P->ev_done[s], cs));
        // outputs
        PIPE_CUDA(cudaStreamWaitEvent(P->out, P->ev_done[s], 0));
        PIPE_CUDA(cudaMemcpyAsync(h_iou + k0, d_iou, (size_t)m * 4, cudaMemcpyDeviceToHost, P->out));
        PIPE_CUDA(cudaMemcpyAsync(h_g1 + (size_t)k0 * K * 2, d_g1, (size_t)m * pp, cudaMemcpyDeviceToHost, P->out));
        PIPE_CUDA(cudaMemcpyAsync(h_g2 + (size_t)k0 * K * 2, d_g2, (size_t)m * pp, cudaMemcpyDeviceToHost, P->out));
        PIPE_CUDA(cudaEventRecord(P->ev_out[s], P->out));
    }
    // the caller's stream ends after the last copies out
    const int64_t first = nchunks > kSlots ? nchunks - kSlots : 0;
    for (int64_t c = first; c < nchunks; ++c) PIPE_CUDA(cudaStreamWaitEvent(cs, P->ev_out[c % kSlots], 0));
    return DGAL_OK;
}
