// Pairwise IoU matrices: one N x M matrix, or a ragged batch of S matrices
// in one persistent launch.
//
// One matrix: tiles of 32 rows x 128 columns; an exact axis-aligned
// bounding-box test (comparisons on the float inputs, no rounding) on every
// entry first, since disjoint pairs have IoU 0 and nx 0 by definition (no
// vertex inside, no crossing), then the clip on the queued entries whose
// boxes meet, densely (see k_pairwise).  Consecutive lanes write consecutive
// IoU floats and nx bytes.
//
// Ragged batch: a setup kernel turns the device-side offsets into a tile
// prefix (tiles of rows x threads entries of one scene's matrix) and resets a
// queue counter; persistent blocks (SMs x blocks_sm) pop tile numbers with
// one atomicAdd each until the queue is empty and run pw_tile on each.  The queue only
// grows, nothing waits on it, so the launch cannot hang; everything it reads
// lives on the device, so the pair of launches can be captured in a graph.
#include "dgal_geom.cuh"
#include "dgal_internal.h"
#include "pw_entry.cuh"

namespace dgal {

// Single matrices narrower than this, or with fewer than two tiles per SM,
// take the one-thread-per-entry kernel (the tiled one would leave most of a
// tile's columns, or most SMs, idle).
constexpr int64_t kFlatMaxCols = 96;

// Rows of a ragged-batch tile: entries per tile / threads, at most this.
constexpr int kMaxTileRows = 32;

// Tiles of the N x M matrix: kTileRows rows x kPwThreads columns.  On the
// 2000 x 2000 bird's-eye matrix, 32 rows measured 26.6 us against 29.4 at 16
// rows and 33.5 at 8 while blocks looped over tiles; with one tile per block,
// 16, 32 and 64 rows measured within 24.6-25.4 us.  More rows give each tile
// more queued entries, so more of its warps clip at once.
constexpr int kTileRows = 32;

// Blocks per SM the K = 4 tile kernel is compiled for (registers <= 65536 /
// (128 x this)); K = 8 holds its polygons in registers and takes 1.  At 7
// (72 registers, a few spills) the 1008 tiles of a 2000 x 2000 matrix fit in
// one wave of 152 x 7 blocks: 21.8 -> 19.8 us against 5; 6 and 8 measured
// 22.4 and 19.9 us.
constexpr int kPwMinBlocks = 7;

// One N x M matrix: one block per tile of kTileRows x kPwThreads entries
// (pw_tile).  Without a loop over tiles the kernel holds fewer registers, so
// more blocks share an SM; the tile count fits a 1-D grid for any matrix whose
// outputs fit in memory.
template <int K, bool COUNTS>
__global__ void __launch_bounds__(kPwThreads, K == 4 ? kPwMinBlocks : 1)
k_pairwise(const float* __restrict__ a, const uint8_t* __restrict__ ca, int64_t N, const float* __restrict__ b,
           const uint8_t* __restrict__ cb, int64_t M, float* __restrict__ iou, uint8_t* __restrict__ nx,
           uint32_t flags, uint32_t* status) {
    __shared__ float4 s_rbox[kTileRows];
    __shared__ uint16_t s_q[kTileRows * kPwThreads];
    __shared__ int s_nq[kPwMaxWarps];
    const bool refine = (flags & kFlagRefine) && !(flags & kFlagPlain);
    const int64_t cblocks = (M + kPwThreads - 1) / kPwThreads;
    const int64_t rb = blockIdx.x / cblocks;
    uint32_t err = 0;
    pw_tile<K, COUNTS>(a, ca, N, b, cb, M, rb * kTileRows, ((int64_t)blockIdx.x - rb * cblocks) * kPwThreads,
                       kTileRows, s_rbox, s_q, s_nq, refine, err, PwMatrixOut{iou, nx, M});
    if (err) atomicOr(status, err);
}

// Small or narrow matrices: one thread per entry, row-major (no tiles, so a
// small matrix still spreads over many blocks).
template <int K, bool COUNTS>
__global__ void __launch_bounds__(kPwThreads)
k_pairwise_flat(const float* __restrict__ a, const uint8_t* __restrict__ ca, int64_t N, const float* __restrict__ b,
           const uint8_t* __restrict__ cb, int64_t M, float* __restrict__ iou, uint8_t* __restrict__ nx,
           uint32_t flags, uint32_t* status) {
    const int lane = threadIdx.x & 31;
    const int64_t total = N * M;
    const int64_t stride = (int64_t)gridDim.x * kPwThreads;
    const bool refine = (flags & kFlagRefine) && !(flags & kFlagPlain);
    int64_t base = (int64_t)blockIdx.x * kPwThreads + (threadIdx.x & ~31);
    if (base >= total) return;
    const int64_t e0 = base + lane;
    int64_t i = e0 / M, j = e0 - (e0 / M) * M;
    const int64_t di = stride / M, dj = stride - di * M;
    uint32_t err = 0;
    for (; base < total; base += stride) {
        const int64_t e = base + lane;
        const bool act = e < total;
        const int n1 = (COUNTS && ca && act) ? (int)ca[i] : K;
        const int n2 = (COUNTS && cb && act) ? (int)cb[j] : K;
        const float* pa = a + (act ? i : 0) * 2 * K;
        const float* pb = b + (act ? j : 0) * 2 * K;
        float v = 0.f;
        uint32_t c = 0;
        const bool hard = act && pw_fast<K, COUNTS>(pa, pb, n1, n2, v, c, err, refine);
        pw_finish<K>(__ballot_sync(0xffffffffu, hard), pa, pb, n1, n2, refine, v, c, err);
        if (act) {
            iou[e] = v;
            if (nx) nx[e] = (uint8_t)c;
        }
        i += di;
        j += dj;
        if (j >= M) {
            j -= M;
            ++i;
        }
    }
    if (err) atomicOr(status, err);
}

// ------------------------------------------------------------ ragged batch

// workspace: [0] uint32 queue counter, [16 B ..] int64 tile_start[S + 1]
size_t batched_workspace_bytes(int S) { return 16 + (((size_t)(S + 1) * 8 + 15) / 16) * 16; }

constexpr int kSetupThreads = 1024;

__global__ void __launch_bounds__(kSetupThreads)
k_batched_setup(int S, const int64_t* __restrict__ a_off, const int64_t* __restrict__ b_off,
                const int64_t* __restrict__ out_off, int64_t rows, int64_t cols, uint32_t* __restrict__ counter,
                int64_t* __restrict__ tile_start, uint32_t* status) {
    __shared__ int64_t part[kSetupThreads];
    const int t = threadIdx.x;
    const int chunk = (S + kSetupThreads - 1) / kSetupThreads;
    const int s0 = t * chunk, s1 = min(S, s0 + chunk);
    int64_t sum = 0;
    uint32_t err = 0;
    for (int s = s0; s < s1; ++s) {
        const int64_t Ns = a_off[s + 1] - a_off[s], Ms = b_off[s + 1] - b_off[s];
        const int64_t E = out_off[s + 1] - out_off[s];
        const bool ok = Ns >= 0 && Ms >= 0 && E == Ns * Ms && a_off[0] == 0 && b_off[0] == 0 && out_off[0] == 0;
        err |= ok ? 0u : kDevBadOffsets;
        sum += ok ? ((Ns + rows - 1) / rows) * ((Ms + cols - 1) / cols) : 0;
    }
    part[t] = sum;
    __syncthreads();
    // inclusive scan over the per-thread sums (Hillis-Steele)
    for (int off = 1; off < kSetupThreads; off <<= 1) {
        int64_t v = (t >= off) ? part[t - off] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int64_t run = part[t] - sum;
    for (int s = s0; s < s1; ++s) {
        tile_start[s] = run;
        const int64_t Ns = a_off[s + 1] - a_off[s], Ms = b_off[s + 1] - b_off[s];
        const int64_t E = out_off[s + 1] - out_off[s];
        const bool ok = Ns >= 0 && Ms >= 0 && E == Ns * Ms && a_off[0] == 0 && b_off[0] == 0 && out_off[0] == 0;
        run += ok ? ((Ns + rows - 1) / rows) * ((Ms + cols - 1) / cols) : 0;
    }
    if (t == kSetupThreads - 1) {
        tile_start[S] = part[t];
        *counter = 0u;
    }
    if (err) atomicOr(status, err);
}

// K = 4: at most 85 registers (3 blocks of 256 or 6 of 128 per SM), 80 in
// practice, so the persistent blocks the tuner asks for stay resident: the
// 64-scene batch went 62.4 -> 58.2 us (the tuner then picks 12 blocks of 128
// per SM instead of 8).
template <int K, bool COUNTS>
__global__ void __launch_bounds__(256, K == 4 ? 3 : 1) k_batched(int S, const int64_t* __restrict__ a_off, const int64_t* __restrict__ b_off,
                          const int64_t* __restrict__ out_off, const float* __restrict__ a,
                          const uint8_t* __restrict__ ca, const float* __restrict__ b, const uint8_t* __restrict__ cb,
                          float* __restrict__ iou, uint8_t* __restrict__ nx, uint32_t* __restrict__ counter,
                          const int64_t* __restrict__ tile_start, int rows, uint32_t flags, uint32_t* status) {
    extern __shared__ uint16_t s_q[]; // rows x blockDim.x queue codes
    __shared__ float4 s_rbox[kMaxTileRows];
    __shared__ int64_t s_tile;
    __shared__ int s_scene;
    __shared__ int s_nq[kPwMaxWarps];
    const bool refine = (flags & kFlagRefine) && !(flags & kFlagPlain);
    const int64_t total = tile_start[S];
    const int64_t cols = blockDim.x;
    uint32_t err = 0;
    for (;;) {
        if (threadIdx.x == 0) {
            const int64_t t = (int64_t)atomicAdd(counter, 1u);
            int lo = 0, hi = S; // largest s with tile_start[s] <= t (tile_start[S] = total > t)
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (tile_start[mid] <= t) lo = mid; else hi = mid;
            }
            s_tile = t;
            s_scene = lo;
        }
        __syncthreads();
        const int64_t t = s_tile;
        const int s = s_scene;
        __syncthreads();
        if (t >= total) break;
        const int64_t a0 = a_off[s], b0 = b_off[s], o0 = out_off[s];
        const int64_t Ns = a_off[s + 1] - a0, Ms = b_off[s + 1] - b0;
        const int64_t cblocks = (Ms + cols - 1) / cols;
        const int64_t lt = t - tile_start[s];
        const int64_t rb = lt / cblocks;
        const PwMatrixOut out{iou + o0, nx ? nx + o0 : nullptr, Ms};
        pw_tile<K, COUNTS>(a + a0 * 2 * K, COUNTS && ca ? ca + a0 : nullptr, Ns, b + b0 * 2 * K,
                           COUNTS && cb ? cb + b0 : nullptr, Ms, rb * rows, (lt - rb * cblocks) * cols, rows, s_rbox,
                           s_q, s_nq, refine, err, out);
    }
    if (err) atomicOr(status, err);
}

template <int K, bool COUNTS>
static void pairwise_dispatch(const float* a, const uint8_t* ca, int64_t N, const float* b, const uint8_t* cb,
                              int64_t M, float* iou, uint8_t* nx, uint32_t flags, cudaStream_t s) {
    const int64_t tiles = ((N + kTileRows - 1) / kTileRows) * ((M + kPwThreads - 1) / kPwThreads);
    if (M < kFlatMaxCols || tiles < (int64_t)sm_count() * 2) {
        // narrow or small: one thread per entry spreads over more blocks
        int64_t blocks = (N * M + kPwThreads - 1) / kPwThreads;
        const int64_t cap = (int64_t)sm_count() * 32;
        if (blocks > cap) blocks = cap;
        k_pairwise_flat<K, COUNTS><<<(unsigned)blocks, kPwThreads, 0, s>>>(a, ca, N, b, cb, M, iou, nx, flags,
                                                                            device_status_ptr());
        return;
    }
    // tiles <= N * M / kPwThreads; an output of 2^31 * 128 entries would not fit in memory
    k_pairwise<K, COUNTS><<<(unsigned)tiles, kPwThreads, 0, s>>>(a, ca, N, b, cb, M, iou, nx, flags,
                                                                  device_status_ptr());
}

dgal_status launch_pairwise(const float* a, const uint8_t* ca, int64_t N, const float* b, const uint8_t* cb,
                            int64_t M, int K, float* iou, uint8_t* nx, uint32_t flags, cudaStream_t s) {
    if (!device_status_ptr()) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    const bool counts = ca || cb;
    if (K == 4) {
        if (counts) pairwise_dispatch<4, true>(a, ca, N, b, cb, M, iou, nx, flags, s);
        else pairwise_dispatch<4, false>(a, ca, N, b, cb, M, iou, nx, flags, s);
    } else {
        if (counts) pairwise_dispatch<8, true>(a, ca, N, b, cb, M, iou, nx, flags, s);
        else pairwise_dispatch<8, false>(a, ca, N, b, cb, M, iou, nx, flags, s);
    }
    return check_launch("pairwise");
}

// Tile shape of the ragged batch: cfg.threads columns x (cfg.tile /
// cfg.threads) rows, 1 to kMaxTileRows.
static int batched_rows(const BatchedConfig& cfg) {
    int r = cfg.tile / (cfg.threads > 0 ? cfg.threads : 1);
    return r < 1 ? 1 : (r > kMaxTileRows ? kMaxTileRows : r);
}

template <int K, bool COUNTS>
static void batched_dispatch(int S, const int64_t* a_off, const int64_t* b_off, const int64_t* out_off,
                             const float* a, const uint8_t* ca, const float* b, const uint8_t* cb, float* iou,
                             uint8_t* nx, uint32_t* counter, const int64_t* tile_start, uint32_t flags,
                             const BatchedConfig& cfg, cudaStream_t s) {
    const unsigned grid = (unsigned)(sm_count() * cfg.blocks_sm);
    const int rows = batched_rows(cfg);
    k_batched<K, COUNTS><<<grid, cfg.threads, (size_t)rows * cfg.threads * sizeof(uint16_t), s>>>(
        S, a_off, b_off, out_off, a, ca, b, cb, iou, nx, counter, tile_start, rows, flags, device_status_ptr());
}

dgal_status launch_batched(int S, const int64_t* a_off, const int64_t* b_off, const int64_t* out_off,
                           const float* a, const uint8_t* ca, const float* b, const uint8_t* cb, int K, float* iou,
                           uint8_t* nx, void* ws, uint32_t flags, const BatchedConfig& cfg, cudaStream_t s) {
    if (!device_status_ptr()) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    uint32_t* counter = static_cast<uint32_t*>(ws);
    int64_t* tile_start = reinterpret_cast<int64_t*>(static_cast<char*>(ws) + 16);
    k_batched_setup<<<1, kSetupThreads, 0, s>>>(S, a_off, b_off, out_off, (int64_t)batched_rows(cfg),
                                                (int64_t)cfg.threads, counter, tile_start, device_status_ptr());
    dgal_status st = check_launch("batched setup");
    if (st != DGAL_OK) return st;
    const bool counts = ca || cb;
    if (K == 4) {
        if (counts) batched_dispatch<4, true>(S, a_off, b_off, out_off, a, ca, b, cb, iou, nx, counter, tile_start, flags, cfg, s);
        else batched_dispatch<4, false>(S, a_off, b_off, out_off, a, ca, b, cb, iou, nx, counter, tile_start, flags, cfg, s);
    } else {
        if (counts) batched_dispatch<8, true>(S, a_off, b_off, out_off, a, ca, b, cb, iou, nx, counter, tile_start, flags, cfg, s);
        else batched_dispatch<8, false>(S, a_off, b_off, out_off, a, ca, b, cb, iou, nx, counter, tile_start, flags, cfg, s);
    }
    return check_launch("batched");
}

} // namespace dgal
