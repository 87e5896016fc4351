// Allocation-free variant of the ragged batched pairwise IoU.
//
// Some callers cannot allocate device memory at the moment they need this
// call: code that runs while a stream is being captured into a CUDA graph
// (an allocation there breaks or pollutes the capture), latency-critical loops
// where cudaMalloc would stall the device, and plugins inside a host framework
// that owns every device allocation itself.  For them the scratch that
// dgal_iou_pairwise_batched normally takes from the caller (a queue counter
// and the per-scene tile prefix) lives here instead, in one fixed array that
// is compiled into the library; every GPU that loads the library holds it until
// the process exits.
#include <map>
#include <mutex>

#include "dgal_internal.h"

namespace dgal {
namespace {

// Largest number of scenes one call accepts; the array holds the queue counter
// (16 bytes) and tile_start[S + 1] as int64, i.e. 16 + 8 * 4097 bytes rounded up.
constexpr int kNoAllocMaxScenes = 4096;
constexpr size_t kNoAllocBytes = 16 + ((size_t)(kNoAllocMaxScenes + 1) * 8 + 15) / 16 * 16;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
std::map<int, void*> g_noalloc_ptr; // device ordinal -> device address of the array

// The array's name in host code is only a host-side handle, so its device
// address is looked up once per device (with that device current) and cached.
dgal_status noalloc_scratch(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return fail(DGAL_ERR_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    auto it = g_noalloc_ptr.find(dev);
    if (it != g_noalloc_ptr.end()) {
        *out = it->second;
        return DGAL_OK;
    }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr)
        return fail(DGAL_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_noalloc_ptr[dev] = p;
    *out = p;
    return DGAL_OK;
}

} // namespace
} // namespace dgal

using namespace dgal;

extern "C" dgal_status dgal_iou_pairwise_batched_noalloc(int S, const int64_t* a_off, const int64_t* b_off,
                                                         const int64_t* out_off, const float* a, const uint8_t* ca,
                                                         const float* b, const uint8_t* cb, int K, float* iou,
                                                         uint8_t* nx, uint32_t flags, void* stream) {
    clear_last_error();
    if (S == 0) return DGAL_OK;
    // the arguments are checked first, so a bad K or pointer is reported as
    // such whatever S is
    if (dgal_status st = check_batched_args(S, a_off, b_off, out_off, a, b, K, iou); st != DGAL_OK) return st;
    if (S > kNoAllocMaxScenes)
        return fail(DGAL_ERR_WORKSPACE,
                    "S = %d scenes exceeds the fixed scratch of dgal_iou_pairwise_batched_noalloc (at most %d); "
                    "use dgal_iou_pairwise_batched with a caller workspace",
                    S, kNoAllocMaxScenes);
    void* ws = nullptr;
    dgal_status st = noalloc_scratch(&ws);
    if (st != DGAL_OK) return st;
    // Same validation and launches as the workspace form; the setup kernel
    // rewrites the counter and the tile prefix on every call.
    return dgal_iou_pairwise_batched(S, a_off, b_off, out_off, a, ca, b, cb, K, iou, nx, ws, kNoAllocBytes, flags,
                                     stream);
}
