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
//   2. k_nms_mask    one block per tile of 32 rows x 128 columns (two 64-bit
//                    words per row) of the visiting-order matrix, on or right
//                    of the rows' diagonal word: the pairwise tile
//                    (pw_entry.cuh: exact box test on every entry b > a, the
//                    same FP32 IoU as dgal_iou_pairwise on the queued ones)
//                    sets bit b of row a's word when IoU(a, b) > thr.  The
//                    tile stores its words and, for the diagonal 64 x 64
//                    block, also its transpose: for each row b, the rows a < b
//                    of its 64-row block that suppress it;
//   3. k_nms_greedy  one block walks the rows 64 at a time.  Warp 0 decides
//                    the block's rows from the transposed diagonal in a few
//                    ballot rounds (a row is kept once none of its
//                    suppressors is kept or undecided, suppressed once one of
//                    them is kept; every round decides at least the lowest
//                    undecided row), then the kept rows' later words are ORed
//                    into the removal bitmap held in shared memory.  What a
//                    64-row block reads (transposed diagonal, visiting order,
//                    the rows' next 32 words) does not depend on the outcome,
//                    so asynchronous copies (cp.async) bring it into a ring of
//                    shared-memory stages kNmsStages - 1 blocks ahead, and the
//                    walk does not wait on memory; words further right are
//                    loaded for kept rows only.
#include <cmath>

#include "dgal_geom.cuh"
#include "dgal_internal.h"
#include "pw_entry.cuh"

namespace dgal {

constexpr int64_t kNmsMaxBoxes = 131072; // removal bitmap: 2048 words = 16 KB of shared memory (+ 67 KB of stages)
constexpr int kNmsThreads = 128;         // rank kernel: 4 warps, one box each
constexpr int kNmsRowsPerBlock = kNmsThreads / 32;
constexpr int kNmsGreedyThreads = 1024;  // 32 warps: warp k holds rows k and k + 32 of a 64-row block

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct NmsLayout {
    size_t order, boxes, counts, mask, sup, total;
};

// Workspace: order int32 [N] | polygons in visiting order float [N][K][2] |
// their counts uint8 [N] | suppression words uint64 [N][W], W = ceil(N / 64) |
// transposed diagonal uint32 [N][2] (word of row b, bit a mod 64: a < b in
// the same 64-row block suppresses b; half h written by the tile of rows
// 64 (b / 64) + 32 h).
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
    L.sup = off;
    off += align256((size_t)N * 8);
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

// Tile output of the suppression mask: bit (b - j0) of the tile's two words
// of row a is set when IoU(a, b) > thr, and for a, b in the same 64-row block
// bit a mod 32 of column b's transposed word.  Only entries right of the
// diagonal are wanted (row a is suppressed by earlier rows only).  Disjoint
// pairs have IoU 0, which exceeds only a negative threshold.
struct NmsBitsOut {
    unsigned long long* bits; // shared memory: 2 words per tile row
    unsigned* tbits;          // shared memory: 1 transposed half-word per tile column
    int64_t i0, j0;
    float thr;
    __device__ __forceinline__ bool wanted(int64_t i, int64_t j) const { return j > i; }
    __device__ __forceinline__ void set(int64_t i, int64_t j) const {
        atomicOr(&bits[(i - i0) * 2 + ((j - j0) >> 6)], 1ull << ((j - j0) & 63));
        if ((i >> 6) == (j >> 6)) atomicOr(&tbits[j - j0], 1u << (i & 31));
    }
    __device__ __forceinline__ void disjoint(int64_t i, int64_t j) const {
        if (0.f > thr) set(i, j);
    }
    __device__ __forceinline__ void put(int64_t i, int64_t j, float v, uint32_t) const {
        if (v > thr) set(i, j);
    }
};

constexpr int kNmsTileRows = 32; // rows of a mask tile; its kPwThreads = 128 columns are two words

template <int K, bool COUNTS>
__global__ void __launch_bounds__(kPwThreads)
k_nms_mask(const float* __restrict__ sboxes, const uint8_t* __restrict__ scounts, int64_t N, int64_t W, float thr,
           uint64_t* __restrict__ mask, uint32_t* __restrict__ sup, uint32_t flags, uint32_t* status) {
    __shared__ float4 s_rbox[kNmsTileRows];
    __shared__ uint16_t s_q[kNmsTileRows * kPwThreads];
    __shared__ int s_nq;
    __shared__ unsigned long long s_bits[kNmsTileRows * 2];
    __shared__ unsigned s_tbits[kPwThreads];
    const int t = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.y * kNmsTileRows, w0 = 2 * (int64_t)blockIdx.x, j0 = w0 * 64;
    // all the tile's rows share the diagonal word i0 / 64 (tiles are 32-row
    // aligned); words left of it are never read
    const int64_t c0 = i0 >> 6;
    if (w0 + 1 < c0) return; // block-uniform
    const bool refine = (flags & kFlagRefine) && !(flags & kFlagPlain);
    // ordered before any put by pw_tile's first barrier
    if (t < kNmsTileRows * 2) s_bits[t] = 0ull;
    s_tbits[t] = 0u;
    uint32_t err = 0;
    const NmsBitsOut out{s_bits, s_tbits, i0, j0, thr};
    pw_tile<K, COUNTS>(sboxes, scounts, N, sboxes, scounts, N, i0, j0, kNmsTileRows, s_rbox, s_q, &s_nq, refine, err,
                       out);
    // pw_tile ends with a barrier: the bits are final
    if (t < kNmsTileRows * 2) {
        const int64_t a = i0 + (t >> 1), w = w0 + (t & 1);
        if (a < N && w < W && w >= c0) mask[a * W + w] = s_bits[t];
    }
    const int64_t j = j0 + t;
    if (j < N && (j >> 6) == c0) sup[j * 2 + ((i0 >> 5) & 1)] = s_tbits[t];
    if (err) atomicOr(status, err);
}

// What the greedy pass reads for one 64-row block: the rows' words
// c + 1 .. c + 32, their transposed diagonal words and their box indices.
struct NmsStage {
    uint64_t near[64][32];
    uint64_t sup[64];
    int32_t ord[64];
};
constexpr int kNmsStages = 4;

__device__ __forceinline__ void cp_async(void* dst, const void* src, int bytes, bool pred) {
    // src-size 0 copies nothing and fills the destination with zeros
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if (bytes == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(d), "l"(src), "r"(pred ? 8 : 0) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(pred ? 4 : 0) : "memory");
}

__global__ void __launch_bounds__(kNmsGreedyThreads)
k_nms_greedy(const int32_t* __restrict__ order, const uint64_t* __restrict__ mask, const uint64_t* __restrict__ sup,
             int64_t N, int64_t W, int64_t* __restrict__ keep, int64_t* __restrict__ num_keep) {
    extern __shared__ __align__(16) unsigned char g_smem[];
    NmsStage* stage = reinterpret_cast<NmsStage*>(g_smem);
    // W words: bit b of word w = row 64 w + b is suppressed
    unsigned long long* removed = reinterpret_cast<unsigned long long*>(g_smem + kNmsStages * sizeof(NmsStage));
    __shared__ uint64_t s_kept;
    __shared__ int s_rows[64]; // the kept rows of the current block, in order
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    for (int64_t w = t; w < W; w += blockDim.x) removed[w] = 0ull;
    // copies of block c into its stage (none past the last block), one group per block
    auto issue = [&](int64_t c) {
        if (c < W) {
            NmsStage& st = stage[c % kNmsStages];
            const int64_t r0 = c * 64 + wp, r1 = r0 + 32, w = c + 1 + lane;
            cp_async(&st.near[wp][lane], (r0 < N && w < W) ? mask + r0 * W + w : mask, 8, r0 < N && w < W);
            cp_async(&st.near[wp + 32][lane], (r1 < N && w < W) ? mask + r1 * W + w : mask, 8, r1 < N && w < W);
            const int64_t r = c * 64 + (t & 63);
            if (t < 64) cp_async(&st.sup[t], r < N ? sup + r : sup, 8, r < N);
            else if (t < 128) cp_async(&st.ord[t - 64], r < N ? order + r : order, 4, r < N);
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    for (int c = 0; c < kNmsStages - 1; ++c) issue(c);
    int64_t count = 0;
    for (int64_t c = 0; c < W; ++c) {
        // block c's group is the oldest of the kNmsStages - 1 in flight
        asm volatile("cp.async.wait_group %0;\n" ::"n"(kNmsStages - 2) : "memory");
        __syncthreads(); // every thread's copies of block c, the removal words, the previous block done
        issue(c + kNmsStages - 1); // into the stage the previous block used
        const NmsStage& st = stage[c % kNmsStages];
        if (wp == 0) {
            const int64_t rows = N - c * 64;
            const uint64_t valid = rows >= 64 ? ~0ull : ((1ull << rows) - 1ull);
            // suppressors of rows 64 c + lane and 64 c + 32 + lane: only bits below the row count
            const uint64_t sb0 = st.sup[lane] & ((1ull << lane) - 1ull);
            const uint64_t sb1 = st.sup[lane + 32] & ((1ull << (lane + 32)) - 1ull);
            uint64_t und = ~removed[c] & valid, kept = 0ull; // warp-uniform
            while (und) {
                const bool u0 = (und >> lane) & 1ull, u1 = (und >> (lane + 32)) & 1ull;
                const uint64_t live = und | kept;
                const uint64_t k = (uint64_t)__ballot_sync(0xffffffffu, u0 && !(sb0 & live)) |
                                   ((uint64_t)__ballot_sync(0xffffffffu, u1 && !(sb1 & live)) << 32);
                const uint64_t x = (uint64_t)__ballot_sync(0xffffffffu, u0 && (sb0 & kept)) |
                                   ((uint64_t)__ballot_sync(0xffffffffu, u1 && (sb1 & kept)) << 32);
                kept |= k;
                und &= ~(k | x);
            }
            if (lane == 0) s_kept = kept;
        }
        __syncthreads();
        const uint64_t kept = s_kept;
        if (t < 64 && ((kept >> t) & 1ull)) {
            const int slot = __popcll(kept & ((1ull << t) - 1ull));
            keep[count + slot] = (int64_t)st.ord[t];
            s_rows[slot] = t;
        }
        const int nk = __popcll(kept);
        count += nk;
        // near words of the kept rows (zero past the last word)
        const uint64_t v = (((kept >> wp) & 1ull) ? st.near[wp][lane] : 0ull) |
                           (((kept >> (wp + 32)) & 1ull) ? st.near[wp + 32][lane] : 0ull);
        if (v) atomicOr(&removed[c + 1 + lane], (unsigned long long)v);
        // words c + 33 .. W - 1: every (kept row, word) pair on its own thread
        const int nfar = (int)(W - c - 33); // W <= 2048: 32-bit indices
        if (nfar > 0) {
            __syncthreads(); // s_rows
            for (int idx = t; idx < nk * nfar; idx += blockDim.x) {
                const int kk = idx / nfar, w = (int)c + 33 + (idx - kk * nfar);
                const uint64_t f = mask[(c * 64 + s_rows[kk]) * W + w];
                if (f) atomicOr(&removed[w], (unsigned long long)f);
            }
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    if (t == 0) *num_keep = count;
}

static size_t nms_greedy_smem(int64_t W) { return kNmsStages * sizeof(NmsStage) + (size_t)W * 8; }

template <int K, bool COUNTS>
static void nms_mask_dispatch(const float* sboxes, const uint8_t* scounts, int64_t N, int64_t W, float thr,
                              uint64_t* mask, uint32_t* sup, uint32_t flags, cudaStream_t s) {
    // x: pairs of words (128 columns), y: 32-row tiles; N <= kNmsMaxBoxes keeps y <= 4096
    const dim3 grid((unsigned)((N + kPwThreads - 1) / kPwThreads), (unsigned)((N + kNmsTileRows - 1) / kNmsTileRows));
    k_nms_mask<K, COUNTS><<<grid, kPwThreads, 0, s>>>(sboxes, scounts, N, W, thr, mask, sup, flags,
                                                       device_status_ptr());
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
    uint32_t* sup = reinterpret_cast<uint32_t*>(base + L.sup);
    const int64_t W = (N + 63) / 64;
    const unsigned rank_grid = (unsigned)((N + kNmsRowsPerBlock - 1) / kNmsRowsPerBlock);
    if (K == 4) k_nms_rank<4><<<rank_grid, kNmsThreads, 0, s>>>(boxes, counts, scores, N, order, sboxes, scounts);
    else k_nms_rank<8><<<rank_grid, kNmsThreads, 0, s>>>(boxes, counts, scores, N, order, sboxes, scounts);
    dgal_status st = check_launch("nms rank");
    if (st != DGAL_OK) return st;
    if (K == 4) {
        if (counts) nms_mask_dispatch<4, true>(sboxes, scounts, N, W, thr, mask, sup, flags, s);
        else nms_mask_dispatch<4, false>(sboxes, scounts, N, W, thr, mask, sup, flags, s);
    } else {
        if (counts) nms_mask_dispatch<8, true>(sboxes, scounts, N, W, thr, mask, sup, flags, s);
        else nms_mask_dispatch<8, false>(sboxes, scounts, N, W, thr, mask, sup, flags, s);
    }
    st = check_launch("nms mask");
    if (st != DGAL_OK) return st;
    const size_t smem = nms_greedy_smem(W);
    cudaError_t e = cudaFuncSetAttribute(k_nms_greedy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail(DGAL_ERR_CUDA, "nms greedy shared memory (%zu bytes): %s", smem, cudaGetErrorString(e));
    k_nms_greedy<<<1, kNmsGreedyThreads, smem, s>>>(order, mask, reinterpret_cast<const uint64_t*>(sup), N, W, keep,
                                                    num_keep);
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
