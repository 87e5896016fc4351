// Rotated non-maximum suppression over convex polygons: the consumer of the
// pairwise IoU matrix in rotated-box detection (the paper's Sec. IV case
// study: rotated boxes whose IoU decides which detections survive).
//
// Greedy NMS visits the boxes by descending score (equal scores: lower index
// first) and keeps a box unless an already kept box overlaps it with
// IoU > threshold.  Three launches, all on the caller's stream:
//   1. k_nms_rank    one warp per box counts the boxes that come before it
//                    (its rank in the visiting order) and copies the polygon
//                    to that slot, so no sort is needed and the order is
//                    deterministic;
//   2. k_nms_mask    one warp per (row a, 64-column word c >= a / 64) of the
//                    visiting-order matrix computes IoU(a, b) for b > a in the
//                    word's 64 columns (pw_entry.cuh, the same FP32 IoU as
//                    dgal_iou_pairwise) and stores the word of bits IoU > thr,
//                    two 32-lane ballots;
//   3. k_nms_greedy  one block walks the words of 64 rows at a time: thread 0
//                    resolves the suppression inside the 64-row block from
//                    its diagonal word, then every (kept row, later word)
//                    pair goes to its own thread, which ORs the word into the
//                    removal bitmap held in shared memory, so the block's
//                    loads are in flight together.  The next diagonal is
//                    fetched while the current rows are applied.  Only kept
//                    rows are ever read.
#include <cmath>

#include "dgal_geom.cuh"
#include "dgal_internal.h"
#include "pw_entry.cuh"

namespace dgal {

constexpr int64_t kNmsMaxBoxes = 131072; // removal bitmap: 2048 words = 16 KB of shared memory
constexpr int kNmsThreads = 128;         // rank and mask kernels: 4 warps, one box / row each
constexpr int kNmsRowsPerBlock = kNmsThreads / 32;
constexpr int kNmsGreedyThreads = 1024;

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct NmsLayout {
    size_t order, boxes, counts, mask, total;
};

// Workspace: order int32 [N] | polygons in visiting order float [N][K][2] |
// their counts uint8 [N] | suppression words uint64 [N][W], W = ceil(N / 64).
static NmsLayout nms_layout(int64_t N, int K) {
    const int64_t W = (N + 63) / 64;
    NmsLayout L;
    size_t off = 0;
    L.order = off;
    off += align256((size_t)N * 4);
    L.boxes = off;
    off += align256((size_t)N * K * 2 * sizeof(float));
    L.counts = off;
    off += align256((size_t)N);
    L.mask = off;
    off += align256((size_t)N * (size_t)W * 8);
    L.total = off;
    return L;
}

// Scores as visiting keys: NaN is visited as -infinity, so the keys with the
// index tie-break form a strict total order and the ranks are a permutation.
__device__ __forceinline__ float nms_key(float s) { return s != s ? -INFINITY : s; }

template <int K>
__global__ void __launch_bounds__(kNmsThreads)
k_nms_rank(const float* __restrict__ boxes, const uint8_t* __restrict__ counts, const float* __restrict__ scores,
           int64_t N, int32_t* __restrict__ order, float* __restrict__ sboxes, uint8_t* __restrict__ scounts) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * kNmsRowsPerBlock + (threadIdx.x >> 5);
    if (i >= N) return; // warp-uniform
    const float si = nms_key(__ldg(scores + i));
    int r = 0;
    for (int64_t j = lane; j < N; j += 32) {
        const float sj = nms_key(__ldg(scores + j));
        r += (sj > si || (sj == si && j < i)) ? 1 : 0;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
    if (lane == 0) order[r] = (int32_t)i;
    if (lane < K / 2)
        reinterpret_cast<float4*>(sboxes)[(int64_t)r * (K / 2) + lane] =
            __ldg(reinterpret_cast<const float4*>(boxes) + i * (K / 2) + lane);
    if (counts && lane == 0) scounts[r] = counts[i];
}

template <int K, bool COUNTS>
__global__ void __launch_bounds__(kNmsThreads)
k_nms_mask(const float* __restrict__ sboxes, const uint8_t* __restrict__ scounts, int64_t N, int64_t W, float thr,
           uint64_t* __restrict__ mask, uint32_t flags, uint32_t* status) {
    const int lane = threadIdx.x & 31;
    const int64_t a = (int64_t)blockIdx.x * kNmsRowsPerBlock + (threadIdx.x >> 5);
    const int64_t c = blockIdx.y;
    if (a >= N || (a >> 6) > c) return; // warp-uniform: words left of the diagonal are never read
    const bool refine = (flags & kFlagRefine) && !(flags & kFlagPlain);
    const int n1 = COUNTS ? (int)scounts[a] : K;
    const float* pa = sboxes + a * 2 * K;
    uint32_t err = 0;
    uint32_t half[2];
#pragma unroll 1
    for (int h = 0; h < 2; ++h) {
        const int64_t b = c * 64 + h * 32 + lane;
        const bool act = b > a && b < N;
        const int n2 = (COUNTS && act) ? (int)scounts[b] : K;
        const float* pb = sboxes + (act ? b : 0) * 2 * K;
        float v = 0.f;
        uint32_t nxv = 0;
        const bool hard = act && pw_fast<K, COUNTS>(pa, pb, n1, n2, v, nxv, err, refine);
        pw_finish<K>(__ballot_sync(0xffffffffu, hard), pa, pb, n1, n2, refine, v, nxv, err);
        half[h] = __ballot_sync(0xffffffffu, act && v > thr);
    }
    if (lane == 0) mask[a * W + c] = (uint64_t)half[0] | ((uint64_t)half[1] << 32);
    if (err) atomicOr(status, err);
}

__global__ void __launch_bounds__(kNmsGreedyThreads)
k_nms_greedy(const int32_t* __restrict__ order, const uint64_t* __restrict__ mask, int64_t N, int64_t W,
             int64_t* __restrict__ keep, int64_t* __restrict__ num_keep) {
    extern __shared__ unsigned long long removed[]; // W words: bit b of word w = row 64 w + b is suppressed
    __shared__ uint64_t diag[2][64];
    __shared__ uint64_t s_kept;
    __shared__ int s_rows[64]; // the kept rows of the current block, in order
    const int t = threadIdx.x;
    for (int64_t w = t; w < W; w += blockDim.x) removed[w] = 0ull;
    if (t < 64) diag[0][t] = (t < N) ? mask[(int64_t)t * W] : 0ull;
    __syncthreads();
    int64_t count = 0;
    for (int64_t c = 0; c < W; ++c) {
        const int buf = (int)(c & 1);
        // the next block's diagonal words do not depend on this block's outcome
        uint64_t nd = 0ull;
        const int64_t rn = (c + 1) * 64 + t;
        if (t < 64 && c + 1 < W && rn < N) nd = mask[rn * W + c + 1];
        if (t == 0) {
            const int64_t rows = N - c * 64;
            const uint64_t valid = rows >= 64 ? ~0ull : ((1ull << rows) - 1ull);
            uint64_t cur = removed[c] | ~valid;
            uint64_t kept = 0ull;
            uint64_t avail = ~cur;
            while (avail) {
                const int r = __ffsll((long long)avail) - 1;
                kept |= 1ull << r;
                cur |= diag[buf][r]; // rows of this block that row r suppresses (all above r)
                avail = (r == 63) ? 0ull : (~cur & (~0ull << (r + 1)));
            }
            s_kept = kept;
        }
        __syncthreads();
        const uint64_t kept = s_kept;
        if (t < 64 && ((kept >> t) & 1ull)) {
            const int slot = __popcll(kept & ((1ull << t) - 1ull));
            keep[count + slot] = (int64_t)order[c * 64 + t];
            s_rows[slot] = t;
        }
        const int nk = __popcll(kept);
        count += nk;
        __syncthreads();
        // every (kept row, later word) pair on its own thread, so all the
        // block's loads are in flight together; shared-memory OR to combine
        const int nw = (int)(W - c - 1), pairs = nk * nw; // W <= 2048: 32-bit indices
        for (int idx = t; idx < pairs; idx += blockDim.x) {
            const int k = idx / nw, w = (int)c + 1 + (idx - k * nw);
            const uint64_t v = mask[(c * 64 + s_rows[k]) * W + w];
            if (v) atomicOr(&removed[w], (unsigned long long)v);
        }
        if (t < 64) diag[buf ^ 1][t] = nd;
        __syncthreads();
    }
    if (t == 0) *num_keep = count;
}

template <int K, bool COUNTS>
static void nms_mask_dispatch(const float* sboxes, const uint8_t* scounts, int64_t N, int64_t W, float thr,
                              uint64_t* mask, uint32_t flags, cudaStream_t s) {
    const dim3 grid((unsigned)((N + kNmsRowsPerBlock - 1) / kNmsRowsPerBlock), (unsigned)W);
    k_nms_mask<K, COUNTS><<<grid, kNmsThreads, 0, s>>>(sboxes, scounts, N, W, thr, mask, flags, device_status_ptr());
}

static dgal_status launch_nms(const float* boxes, const uint8_t* counts, const float* scores, int64_t N, int K,
                              float thr, int64_t* keep, int64_t* num_keep, void* ws, uint32_t flags,
                              cudaStream_t s) {
    if (!device_status_ptr()) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    const NmsLayout L = nms_layout(N, K);
    char* base = static_cast<char*>(ws);
    int32_t* order = reinterpret_cast<int32_t*>(base + L.order);
    float* sboxes = reinterpret_cast<float*>(base + L.boxes);
    uint8_t* scounts = reinterpret_cast<uint8_t*>(base + L.counts);
    uint64_t* mask = reinterpret_cast<uint64_t*>(base + L.mask);
    const int64_t W = (N + 63) / 64;
    const unsigned rank_grid = (unsigned)((N + kNmsRowsPerBlock - 1) / kNmsRowsPerBlock);
    if (K == 4) k_nms_rank<4><<<rank_grid, kNmsThreads, 0, s>>>(boxes, counts, scores, N, order, sboxes, scounts);
    else k_nms_rank<8><<<rank_grid, kNmsThreads, 0, s>>>(boxes, counts, scores, N, order, sboxes, scounts);
    dgal_status st = check_launch("nms rank");
    if (st != DGAL_OK) return st;
    if (K == 4) {
        if (counts) nms_mask_dispatch<4, true>(sboxes, scounts, N, W, thr, mask, flags, s);
        else nms_mask_dispatch<4, false>(sboxes, scounts, N, W, thr, mask, flags, s);
    } else {
        if (counts) nms_mask_dispatch<8, true>(sboxes, scounts, N, W, thr, mask, flags, s);
        else nms_mask_dispatch<8, false>(sboxes, scounts, N, W, thr, mask, flags, s);
    }
    st = check_launch("nms mask");
    if (st != DGAL_OK) return st;
    k_nms_greedy<<<1, kNmsGreedyThreads, (size_t)W * 8, s>>>(order, mask, N, W, keep, num_keep);
    return check_launch("nms greedy");
}

} // namespace dgal

using namespace dgal;

extern "C" size_t dgal_nms_workspace_bytes(int64_t N, int K) {
    if ((K != 4 && K != 8) || N < 0 || N > kNmsMaxBoxes) return 0;
    return nms_layout(N, K).total;
}

extern "C" dgal_status dgal_nms_rotated(const float* boxes, const uint8_t* counts, const float* scores, int64_t N,
                                        int K, float threshold, int64_t* keep, int64_t* num_keep, void* workspace,
                                        size_t ws_bytes, uint32_t flags, void* stream) {
    if (K != 4 && K != 8) return fail(DGAL_ERR_UNSUPPORTED_K, "K = %d is not supported (K must be 4 or 8)", K);
    if (N < 0) return fail(DGAL_ERR_INVALID_ARG, "N = %lld is negative", (long long)N);
    if (N > kNmsMaxBoxes)
        return fail(DGAL_ERR_INVALID_ARG, "N = %lld boxes exceeds the NMS limit of %lld", (long long)N,
                    (long long)kNmsMaxBoxes);
    if (!num_keep) return fail(DGAL_ERR_INVALID_ARG, "num_keep is NULL");
    if (reinterpret_cast<uintptr_t>(num_keep) & 7u) return fail(DGAL_ERR_ALIGNMENT, "num_keep is not 8-byte aligned");
    cudaStream_t s = (cudaStream_t)stream;
    if (N == 0) {
        cudaError_t e = cudaMemsetAsync(num_keep, 0, sizeof(int64_t), s);
        if (e != cudaSuccess) return fail(DGAL_ERR_CUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
        return DGAL_OK;
    }
    if (!boxes) return fail(DGAL_ERR_INVALID_ARG, "boxes is NULL");
    if (reinterpret_cast<uintptr_t>(boxes) & 15u) return fail(DGAL_ERR_ALIGNMENT, "boxes is not 16-byte aligned");
    if (!scores) return fail(DGAL_ERR_INVALID_ARG, "scores is NULL");
    if (reinterpret_cast<uintptr_t>(scores) & 3u) return fail(DGAL_ERR_ALIGNMENT, "scores is not 4-byte aligned");
    if (!keep) return fail(DGAL_ERR_INVALID_ARG, "keep is NULL");
    if (reinterpret_cast<uintptr_t>(keep) & 7u) return fail(DGAL_ERR_ALIGNMENT, "keep is not 8-byte aligned");
    if (!workspace) return fail(DGAL_ERR_WORKSPACE, "workspace is NULL");
    if (reinterpret_cast<uintptr_t>(workspace) & 15u)
        return fail(DGAL_ERR_ALIGNMENT, "workspace is not 16-byte aligned");
    const size_t need = nms_layout(N, K).total;
    if (ws_bytes < need)
        return fail(DGAL_ERR_WORKSPACE, "workspace of %zu bytes is smaller than the %zu bytes needed", ws_bytes, need);
    return launch_nms(boxes, counts, scores, N, K, threshold, keep, num_keep, workspace, flags, s);
}
