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
//                    so the tensor-memory-access engine brings it into a ring
//                    of shared-memory stages kNmsStages - 1 blocks ahead (one
//                    2-D tiled load of 64 rows x 34 words, two 1-D bulk
//                    copies, completion counted on an mbarrier per stage), and
//                    the walk does not wait on memory; words further right are
//                    loaded for kept rows only.
#include <cmath>
#include <mutex>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "dgal_geom.cuh"
#include "dgal_internal.h"
#include "pw_entry.cuh"

namespace dgal {

constexpr int64_t kNmsMaxBoxes = 131072; // removal bitmap: 2048 words = 16 KB of shared memory (+ 71 KB of stages)
constexpr int kNmsThreads = 128;         // rank kernel: 4 warps, one box each
constexpr int kNmsRowsPerBlock = kNmsThreads / 32;
constexpr int kNmsGreedyThreads = 512;   // warp k handles rows k, k + warps, ... of a 64-row block
constexpr int kNmsGreedyWarps = kNmsGreedyThreads / 32;
static_assert(kNmsGreedyThreads >= 128 && 64 % kNmsGreedyWarps == 0, "greedy block shape");

static size_t align256(size_t x) { return (x + 255) / 256 * 256; }

struct NmsLayout {
    size_t order, boxes, counts, mask, sup, total;
};

// Words per row of the suppression matrix, padded to even so that rows and
// even word offsets are 16-byte aligned (bulk copies).
static int64_t nms_row_words(int64_t N) {
    const int64_t W = (N + 63) / 64;
    return W + (W & 1);
}

// Workspace: order int32 [N] | polygons in visiting order float [N][K][2] |
// their counts uint8 [N] | suppression words uint64 [N][Wp], Wp = row words
// (the first ceil(N / 64) used) |
// transposed diagonal uint32 [N][2] (word of row b, bit a mod 64: a < b in
// the same 64-row block suppresses b; half h written by the tile of rows
// 64 (b / 64) + 32 h).
static NmsLayout nms_layout(int64_t N, int K) {
    NmsLayout L;
    size_t off = 0;
    L.order = off;
    off += align256((size_t)N * 4);
    L.boxes = off;
    off += align256((size_t)N * K * 2 * sizeof(float));
    L.counts = off;
    off += align256((size_t)N);
    L.mask = off;
    off += align256((size_t)N * (size_t)nms_row_words(N) * 8);
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
#pragma unroll 4
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
k_nms_mask(const float* __restrict__ sboxes, const uint8_t* __restrict__ scounts, int64_t N, int64_t W, int64_t Wp,
           float thr, uint64_t* __restrict__ mask, uint32_t* __restrict__ sup, uint32_t flags, uint32_t* status) {
    __shared__ float4 s_rbox[kNmsTileRows];
    __shared__ uint16_t s_q[kNmsTileRows * kPwThreads];
    __shared__ int s_nq[kPwMaxWarps];
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
    pw_tile<K, COUNTS>(sboxes, scounts, N, sboxes, scounts, N, i0, j0, kNmsTileRows, s_rbox, s_q, s_nq, refine, err,
                       out);
    // pw_tile ends with a barrier: the bits are final
    if (t < kNmsTileRows * 2) {
        const int64_t a = i0 + (t >> 1), w = w0 + (t & 1);
        if (a < N && w < W && w >= c0) mask[a * Wp + w] = s_bits[t];
    }
    const int64_t j = j0 + t;
    if (j < N && (j >> 6) == c0) sup[j * 2 + ((i0 >> 5) & 1)] = s_tbits[t];
    if (err) atomicOr(status, err);
}

// What the greedy pass reads for one 64-row block c: the rows' words
// s .. s + nb - 1 (s = c + 1 rounded down to even, nb = min(34, Wp), so the
// words c + 1 .. c + 32), packed [row][nb] as the tiled load writes them,
// their transposed diagonal words and their box indices.
constexpr int kNmsNear = 34;
struct NmsStage {
    uint64_t near[64 * kNmsNear];
    uint64_t sup[64];
    int32_t ord[64];
};
static_assert(sizeof(NmsStage) % 128 == 0 && (kNmsNear * 8) % 16 == 0, "tiled-load alignment");
constexpr int kNmsStages = 4;
// Bound on an mbarrier wait, in non-blocking polls (tens of cycles each, so
// well under a second at GB300 clocks); then DGAL_DEV_TIMEOUT.
constexpr int kNmsWaitSpins = 1 << 24;

// Box of the tiled load: words per row (even, >= 2: 16-byte rows) and rows.
__host__ __device__ __forceinline__ int nms_box_words(int64_t Wp) { return Wp < kNmsNear ? (int)Wp : kNmsNear; }
__host__ __device__ __forceinline__ int nms_box_rows(int64_t N) { return N < 64 ? (int)N : 64; }

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

// One bulk copy (global -> this CTA's shared memory) that signals its bytes on `bar`.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

// One 2-D tiled load of the box at (x = word, y = row) that signals its bytes on `bar`.
__device__ __forceinline__ void tiled_load(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::
            "r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
        : "memory");
}

// Waits for the phase of `bar` with the given parity; false after kNmsWaitSpins
// polls.  test_wait never suspends the thread, so the bound is a number of
// polls rather than a number of system-dependent suspend intervals.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
    const unsigned a = smem_addr(bar);
    for (int i = 0; i < kNmsWaitSpins; ++i) {
        unsigned done;
        asm volatile("{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
                     : "=r"(done)
                     : "r"(a), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    return false;
}

__global__ void __launch_bounds__(kNmsGreedyThreads)
k_nms_greedy(const __grid_constant__ CUtensorMap mask_map, const int32_t* __restrict__ order,
             const uint64_t* __restrict__ mask, const uint64_t* __restrict__ sup, int64_t N, int64_t W, int64_t Wp,
             int64_t* __restrict__ keep, int64_t* __restrict__ num_keep, uint32_t* status, int64_t expire_at) {
    extern __shared__ unsigned char g_smem[];
    // stages on a 128-byte boundary (tiled loads); the launch adds 128 bytes for this
    unsigned char* base = g_smem + ((128u - (smem_addr(g_smem) & 127u)) & 127u);
    NmsStage* stage = reinterpret_cast<NmsStage*>(base);
    // W words: bit b of word w = row 64 w + b is suppressed
    unsigned long long* removed = reinterpret_cast<unsigned long long*>(base + kNmsStages * sizeof(NmsStage));
    __shared__ __align__(8) uint64_t s_bar[kNmsStages]; // one transaction barrier per stage
    __shared__ uint64_t s_kept;
    __shared__ int s_rows[64];                             // the kept rows of the current block, in order
    __shared__ uint64_t s_part[kNmsGreedyWarps][32];       // per warp: OR of its kept rows' words c + 1 + lane
    const int t = threadIdx.x, lane = t & 31, wp = t >> 5;
    for (int64_t w = t; w < W; w += blockDim.x) removed[w] = 0ull;
    if (t == 0) {
        for (int i = 0; i < kNmsStages; ++i)
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&s_bar[i])) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    // thread 32 (warp 1) loads block c into its stage: the rows' word window
    // (tiled load; rows past N and words past Wp read as zero), the
    // transposed diagonal words and the box indices (bulk copies, sizes
    // rounded up to 16 bytes into the workspace padding), after arming the
    // stage's barrier with the byte count.
    const int nb = nms_box_words(Wp), br = nms_box_rows(N);
    auto issue = [&](int64_t c) {
        if (t != 32 || c >= W) return;
        NmsStage& st = stage[c % kNmsStages];
        uint64_t* bar = &s_bar[c % kNmsStages];
        const int rows = N - c * 64 < 64 ? (int)(N - c * 64) : 64;
        const unsigned sup_bytes = (unsigned)((rows * 8 + 15) & ~15), ord_bytes = (unsigned)((rows * 4 + 15) & ~15);
        const unsigned total = (unsigned)(nb * br * 8) + sup_bytes + ord_bytes;
        // the stage's previous (generic) reads, ordered by the block barrier, come before these async writes
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(total)
                     : "memory");
        tiled_load(st.near, &mask_map, (int)((c + 1) & ~1ll), (int)(c * 64), bar);
        bulk_copy(st.sup, sup + c * 64, sup_bytes, bar);
        bulk_copy(st.ord, order + c * 64, ord_bytes, bar);
    };
    for (int c = 0; c < kNmsStages - 1; ++c) issue(c);
    int64_t count = 0;
    for (int64_t c = 0; c < W; ++c) {
        // block c's copies landed; every thread waits so that it sees them
        const bool landed = mbar_wait(&s_bar[c % kNmsStages], (unsigned)((c / kNmsStages) & 1));
        // expire_at (tests only): this block's wait is taken as expired once
        // its copies have landed, to run the expiry path without a real stall
        const bool ok = landed && c != expire_at;
        if (__syncthreads_or(!ok)) { // also: the removal words and the previous block are done
            // Expiry: no copy may land in this block's shared memory after it
            // exits, so the copies already issued (blocks c .. c + stages - 2)
            // are waited for, each again within the bound, before the barriers
            // are invalidated and the pass stops with DGAL_DEV_TIMEOUT.
            const int64_t last = (c + kNmsStages - 2 < W - 1) ? c + kNmsStages - 2 : W - 1;
            bool drained = true;
            for (int64_t cc = c; cc <= last; ++cc)
                drained &= mbar_wait(&s_bar[cc % kNmsStages], (unsigned)((cc / kNmsStages) & 1));
            __syncthreads();
            if (t == 0) {
                if (drained)
                    for (int i = 0; i < kNmsStages; ++i)
                        asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(smem_addr(&s_bar[i])) : "memory");
                atomicOr(status, kDevTimeout);
            }
            break;
        }
        issue(c + kNmsStages - 1); // into the stage the previous block used
        const NmsStage& st = stage[c % kNmsStages];
        if (wp == 0) {
            // the previous block's near words: word c + lane gathers the warps' parts
            // (far words of earlier blocks, ORed atomically, are all >= c + 32)
            if (c > 0 && c + lane < W) {
                uint64_t v = 0ull;
#pragma unroll
                for (int k = 0; k < kNmsGreedyWarps; ++k) v |= s_part[k][lane];
                removed[c + lane] |= v;
            }
            __syncwarp();
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
        // near words of the kept rows (word c + 1 + lane is window slot c + 1 + lane - s),
        // per warp; warp 0 ORs the parts into the removal words at the next block
        const int64_t wn = c + 1 + lane;
        if (wn < W) {
            const int slot = (int)(wn - ((c + 1) & ~1ll));
            uint64_t v = 0ull;
#pragma unroll
            for (int q = wp; q < 64; q += kNmsGreedyWarps) v |= ((kept >> q) & 1ull) ? st.near[q * nb + slot] : 0ull;
            s_part[wp][lane] = v;
        }
        // words c + 33 .. W - 1: every (kept row, word) pair on its own thread
        const int nfar = (int)(W - c - 33); // W <= 2048: 32-bit indices
        if (nfar > 0) {
            __syncthreads(); // s_rows
            for (int idx = t; idx < nk * nfar; idx += blockDim.x) {
                const int kk = idx / nfar, w = (int)c + 33 + (idx - kk * nfar);
                const uint64_t f = mask[(c * 64 + s_rows[kk]) * Wp + w];
                if (f) atomicOr(&removed[w], (unsigned long long)f);
            }
        }
    }
    if (t == 0) *num_keep = count;
}

static size_t nms_greedy_smem(int64_t W) { return 128 + kNmsStages * sizeof(NmsStage) + (size_t)W * 8; }

// Tensor map of the suppression matrix for the greedy pass's tiled loads:
// uint64 [N][Wp], box nms_box_words(Wp) x nms_box_rows(N), no swizzle,
// out-of-range elements read as zero.  The encoder is the driver's, found
// through the runtime once.
static dgal_status nms_mask_map(CUtensorMap* map, const uint64_t* mask, int64_t N, int64_t Wp) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    });
    if (!encode) return fail(DGAL_ERR_CUDA, "cuTensorMapEncodeTiled is unavailable");
    const cuuint64_t dims[2] = {(cuuint64_t)Wp, (cuuint64_t)N};
    const cuuint64_t strides[1] = {(cuuint64_t)Wp * 8};
    const cuuint32_t box[2] = {(cuuint32_t)nms_box_words(Wp), (cuuint32_t)nms_box_rows(N)};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_UINT64, 2, const_cast<uint64_t*>(mask), dims, strides, box,
                              estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_NONE, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(DGAL_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return DGAL_OK;
}

template <int K, bool COUNTS>
static void nms_mask_dispatch(const float* sboxes, const uint8_t* scounts, int64_t N, int64_t W, int64_t Wp,
                              float thr, uint64_t* mask, uint32_t* sup, uint32_t flags, cudaStream_t s) {
    // x: pairs of words (128 columns), y: 32-row tiles; N <= kNmsMaxBoxes keeps y <= 4096
    const dim3 grid((unsigned)((N + kPwThreads - 1) / kPwThreads), (unsigned)((N + kNmsTileRows - 1) / kNmsTileRows));
    k_nms_mask<K, COUNTS><<<grid, kPwThreads, 0, s>>>(sboxes, scounts, N, W, Wp, thr, mask, sup, flags,
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
    const int64_t W = (N + 63) / 64, Wp = nms_row_words(N);
    const unsigned rank_grid = (unsigned)((N + kNmsRowsPerBlock - 1) / kNmsRowsPerBlock);
    if (K == 4) k_nms_rank<4><<<rank_grid, kNmsThreads, 0, s>>>(boxes, counts, scores, N, order, sboxes, scounts);
    else k_nms_rank<8><<<rank_grid, kNmsThreads, 0, s>>>(boxes, counts, scores, N, order, sboxes, scounts);
    dgal_status st = check_launch("nms rank");
    if (st != DGAL_OK) return st;
    if (K == 4) {
        if (counts) nms_mask_dispatch<4, true>(sboxes, scounts, N, W, Wp, thr, mask, sup, flags, s);
        else nms_mask_dispatch<4, false>(sboxes, scounts, N, W, Wp, thr, mask, sup, flags, s);
    } else {
        if (counts) nms_mask_dispatch<8, true>(sboxes, scounts, N, W, Wp, thr, mask, sup, flags, s);
        else nms_mask_dispatch<8, false>(sboxes, scounts, N, W, Wp, thr, mask, sup, flags, s);
    }
    st = check_launch("nms mask");
    if (st != DGAL_OK) return st;
    const size_t smem = nms_greedy_smem(W);
    cudaError_t e = cudaFuncSetAttribute(k_nms_greedy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return fail(DGAL_ERR_CUDA, "nms greedy shared memory (%zu bytes): %s", smem, cudaGetErrorString(e));
    CUtensorMap map;
    st = nms_mask_map(&map, mask, N, Wp);
    if (st != DGAL_OK) return st;
    // DGAL_TEST_EXPIRE_WAIT: the expiry path at the second block (or the first when there is one)
    const int64_t expire_at = (flags & DGAL_TEST_EXPIRE_WAIT) ? (W > 1 ? 1 : 0) : -1;
    k_nms_greedy<<<1, kNmsGreedyThreads, smem, s>>>(map, order, mask, reinterpret_cast<const uint64_t*>(sup), N, W,
                                                    Wp, keep, num_keep, device_status_ptr(), expire_at);
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
