// The GIoU and DIoU terms of the IoU loss over convex polygons (the IoU-loss
// case study of the paper, Sec. IV-A, with its generalized and
// distance-penalised forms):
//   GIoU loss term  w (1 - IoU + (A_h - U) / A_h),  A_h the area of the convex
//                   hull of both polygons' vertices, U = A_1 + A_2 - A_i;
//   DIoU loss term  w (1 - IoU + rho2 / c2),  rho2 the squared distance of the
//                   two polygons' vertex means, c2 the squared diameter of the
//                   hull (the largest squared distance of two vertices).
// The IoU part runs in the paired loss kernels; these kernels add the rest.
// The forward pass adds scale w (1 - U / A_h) or scale w rho2 / c2 to its
// own per-warp partials (folded with the IoU partials in a fixed order) and,
// for GIoU, keeps A_h per pair for the backward, whose IoU part then adds
// scale w dloss / A_h to dL/dA_i and subtracts it from dL/dA_1, dL/dA_2 (the
// dependence of -U / A_h on the three areas).  The backward pass here adds
// the remaining terms to the gradients: for GIoU the hull area's shoelace
// adjoint times scale w dloss U / A_h^2, for DIoU the adjoints of rho2 and
// c2.  The forward keeps the hull's vertex order per pair (GIoU), so the
// backward does not wrap the points again.  A pair with U <= 0 has no extra term (and no gradient), as its IoU.
//
// One thread per pair.  The n1 + n2 points sit in shared memory (point v of
// thread t at v * blockDim + t, so a warp's reads of one point index are
// conflict-free), in the frame whose origin is P1's vertex 0.  The hull is
// found by gift wrapping from the lowest point: each step takes the point
// that no other point is to the right of, the farthest one among collinear
// points, and exact duplicates are skipped; at most n1 + n2 steps.  The
// diameter is the first largest pair in index order (P1's vertices, then
// P2's).
#include "dgal_geom.cuh"
#include "dgal_internal.h"

namespace dgal {
namespace {

constexpr int kVarThreads = 128;

template <int K> struct VarPts {
    float x[2 * K][kVarThreads];
    float y[2 * K][kVarThreads];
};

// Loads pair k's points into the thread's column of s (local frame); returns
// n1 + n2 (0 for a count outside [3, K]).
template <int K>
__device__ __forceinline__ int load_points(const float* __restrict__ p1, const uint8_t* __restrict__ c1,
                                           const float* __restrict__ p2, const uint8_t* __restrict__ c2, int64_t k,
                                           VarPts<K>& s, int& n1, int& n2) {
    const int t = threadIdx.x;
    n1 = c1 ? (int)c1[k] : K;
    n2 = c2 ? (int)c2[k] : K;
    if (n1 < 3 || n1 > K || n2 < 3 || n2 > K) return 0;
    float px[K], py[K], qx[K], qy[K];
    load_poly<K>(p1 + k * 2 * K, px, py);
    load_poly<K>(p2 + k * 2 * K, qx, qy);
    const float ox = px[0], oy = py[0];
#pragma unroll
    for (int v = 0; v < K; ++v) {
        if (v < n1) {
            s.x[v][t] = v ? px[v] - ox : 0.f;
            s.y[v][t] = v ? py[v] - oy : 0.f;
        }
    }
#pragma unroll
    for (int v = 0; v < K; ++v) {
        if (v < n2) {
            s.x[n1 + v][t] = qx[v] - ox;
            s.y[n1 + v][t] = qy[v] - oy;
        }
    }
    return n1 + n2;
}

// Counter-clockwise hull of the m points of this thread: returns twice its
// area; order receives the hull's point indices, 4 bits each, h the count.
template <int K>
__device__ __forceinline__ float hull(const VarPts<K>& s, int m, uint64_t& order, int& h) {
    const int t = threadIdx.x;
    int st = 0;
    for (int r = 1; r < m; ++r) {
        const float yr = s.y[r][t], ys = s.y[st][t];
        if (yr < ys || (yr == ys && s.x[r][t] < s.x[st][t])) st = r;
    }
    const float xs = s.x[st][t], ys = s.y[st][t];
    int cur = st;
    float area2 = 0.f;
    order = 0;
    h = 0;
    for (int it = 0; it < m; ++it) {
        const float xc = s.x[cur][t], yc = s.y[cur][t];
        int nxt = -1;
        float nx_ = 0.f, ny_ = 0.f;
        for (int r = 0; r < m; ++r) {
            const float xr = s.x[r][t], yr = s.y[r][t];
            if (xr == xc && yr == yc) continue; // cur itself, or a copy of it
            if (nxt < 0) {
                nxt = r;
                nx_ = xr;
                ny_ = yr;
                continue;
            }
            const float o = (nx_ - xc) * (yr - yc) - (ny_ - yc) * (xr - xc);
            bool take = o < 0.f;
            if (o == 0.f) { // collinear with the candidate: the farther one
                const float dr = (xr - xc) * (xr - xc) + (yr - yc) * (yr - yc);
                const float dn = (nx_ - xc) * (nx_ - xc) + (ny_ - yc) * (ny_ - yc);
                take = dr > dn;
            }
            if (take) {
                nxt = r;
                nx_ = xr;
                ny_ = yr;
            }
        }
        if (nxt < 0) break; // every point coincides
        order |= (uint64_t)cur << (4 * h);
        ++h;
        // shoelace about the start point (small products)
        area2 += (xc - xs) * (ny_ - ys) - (yc - ys) * (nx_ - xs);
        cur = nxt;
        if (nx_ == xs && ny_ == ys) break;
    }
    return area2;
}

// Vertex means' difference (dmx, dmy) and its squared length rho2.
template <int K>
__device__ __forceinline__ void centre(const VarPts<K>& s, int n1, int n2, float& rho2, float& dmx, float& dmy) {
    const int t = threadIdx.x;
    float sx1 = 0.f, sy1 = 0.f, sx2 = 0.f, sy2 = 0.f;
    for (int v = 0; v < n1; ++v) {
        sx1 += s.x[v][t];
        sy1 += s.y[v][t];
    }
    for (int v = 0; v < n2; ++v) {
        sx2 += s.x[n1 + v][t];
        sy2 += s.y[n1 + v][t];
    }
    dmx = sx1 / (float)n1 - sx2 / (float)n2;
    dmy = sy1 / (float)n1 - sy2 / (float)n2;
    rho2 = dmx * dmx + dmy * dmy;
}

// Squared distance of points a and b.
template <int K> __device__ __forceinline__ float dist2(const VarPts<K>& s, int a, int b) {
    const int t = threadIdx.x;
    const float dx = s.x[a][t] - s.x[b][t], dy = s.y[a][t] - s.y[b][t];
    return dx * dx + dy * dy;
}

// The squared diameter of the m points (the first largest pair in index order).
template <int K> __device__ __forceinline__ void diameter(const VarPts<K>& s, int m, float& c2, int& da, int& db) {
    c2 = -1.f;
    da = db = 0;
    for (int a = 0; a < m; ++a) {
        for (int b = a + 1; b < m; ++b) {
            const float d = dist2<K>(s, a, b);
            if (d > c2) {
                c2 = d;
                da = a;
                db = b;
            }
        }
    }
}

// VAR 1: GIoU, 2: DIoU.  u: U per pair from the IoU forward; ah (GIoU):
// receives A_h per pair (+inf when the hull has no area, so that the IoU
// backward adds nothing); aux (GIoU): two words per pair for the backward,
// the hull order (4 bits a point) and its count, so that the backward does
// not wrap the points again.  (DIoU's diameter search over at most 120 point
// pairs costs less than storing and reloading its result: measured.)
template <int K, int VAR>
__global__ void __launch_bounds__(kVarThreads)
k_loss_var_fwd(const float* __restrict__ p1, const uint8_t* __restrict__ c1, const float* __restrict__ p2,
               const uint8_t* __restrict__ c2, int64_t n, const float* __restrict__ weight, float scale,
               const float* __restrict__ u, float* __restrict__ ah, uint64_t* __restrict__ aux,
               float* __restrict__ partials) {
    __shared__ VarPts<K> s;
    float acc = 0.f;
    const int64_t stride = (int64_t)gridDim.x * kVarThreads;
    for (int64_t k = (int64_t)blockIdx.x * kVarThreads + threadIdx.x; k < n; k += stride) {
        int n1, n2;
        const int m = load_points<K>(p1, c1, p2, c2, k, s, n1, n2);
        const float U = __ldg(u + k);
        const float sw = scale * (weight ? __ldg(weight + k) : 1.f);
        if constexpr (VAR == 1) {
            float A = 0.f;
            if (m) {
                uint64_t order;
                int h;
                A = 0.5f * hull<K>(s, m, order, h);
                aux[2 * k] = order;
                aux[2 * k + 1] = (uint64_t)h;
            }
            const bool use = m && U > 0.f && A > 0.f;
            if (use) acc += sw * (1.f - U / A);
            ah[k] = use ? A : __int_as_float(0x7f800000);
        } else {
            if (m && U > 0.f) {
                float rho2, dmx, dmy, c2v;
                int da, db;
                centre<K>(s, n1, n2, rho2, dmx, dmy);
                diameter<K>(s, m, c2v, da, db);
                if (c2v > 0.f) acc += sw * (rho2 / c2v);
            }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if ((threadIdx.x & 31) == 0) partials[((int64_t)blockIdx.x * kVarThreads + threadIdx.x) >> 5] = acc;
}

// Adds the extra terms' gradients to g1, g2 (float [n][K][2], already holding
// the IoU part).  dloss: device pointer to the upstream gradient or NULL (1).
template <int K, int VAR>
__global__ void __launch_bounds__(kVarThreads)
k_loss_var_bwd(const float* __restrict__ p1, const uint8_t* __restrict__ c1, const float* __restrict__ p2,
               const uint8_t* __restrict__ c2, int64_t n, const float* __restrict__ weight, float scale,
               const float* __restrict__ dloss, const float* __restrict__ u, const float* __restrict__ ah,
               const uint64_t* __restrict__ aux, float* __restrict__ g1, float* __restrict__ g2) {
    __shared__ VarPts<K> s;
    __shared__ float gx[2 * K][kVarThreads], gy[2 * K][kVarThreads];
    const int t = threadIdx.x;
    const float dl = dloss ? __ldg(dloss) : 1.f;
    const int64_t stride = (int64_t)gridDim.x * kVarThreads;
    for (int64_t k = (int64_t)blockIdx.x * kVarThreads + threadIdx.x; k < n; k += stride) {
        int n1, n2;
        const int m = load_points<K>(p1, c1, p2, c2, k, s, n1, n2);
        const float U = __ldg(u + k);
        if (!m || !(U > 0.f)) continue;
        const float sw = scale * dl * (weight ? __ldg(weight + k) : 1.f);
        for (int v = 0; v < m; ++v) gx[v][t] = gy[v][t] = 0.f;
        bool any = false;
        if constexpr (VAR == 1) {
            const float A = __ldg(ah + k);
            if (A > 0.f && A < __int_as_float(0x7f800000)) {
                const uint64_t order = __ldg(aux + 2 * k);
                const int h = (int)__ldg(aux + 2 * k + 1);
                const float gh = sw * U / (A * A);
                for (int q = 0; q < h; ++q) {
                    const int c = (int)((order >> (4 * q)) & 15u);
                    const int pv = (int)((order >> (4 * ((q + h - 1) % h))) & 15u);
                    const int nv = (int)((order >> (4 * ((q + 1) % h))) & 15u);
                    gx[c][t] += 0.5f * gh * (s.y[nv][t] - s.y[pv][t]);
                    gy[c][t] += 0.5f * gh * (s.x[pv][t] - s.x[nv][t]);
                }
                any = h >= 3;
            }
        } else {
            float rho2, dmx, dmy;
            centre<K>(s, n1, n2, rho2, dmx, dmy);
            float c2v;
            int da, db;
            diameter<K>(s, m, c2v, da, db);
            if (c2v > 0.f) {
                const float gr = sw / c2v, gc = -sw * rho2 / (c2v * c2v);
                const float ax = 2.f * gr * dmx / (float)n1, ay = 2.f * gr * dmy / (float)n1;
                const float bx = -2.f * gr * dmx / (float)n2, by = -2.f * gr * dmy / (float)n2;
                for (int v = 0; v < n1; ++v) {
                    gx[v][t] = ax;
                    gy[v][t] = ay;
                }
                for (int v = 0; v < n2; ++v) {
                    gx[n1 + v][t] = bx;
                    gy[n1 + v][t] = by;
                }
                const float ex = 2.f * gc * (s.x[da][t] - s.x[db][t]), ey = 2.f * gc * (s.y[da][t] - s.y[db][t]);
                gx[da][t] += ex;
                gy[da][t] += ey;
                gx[db][t] -= ex;
                gy[db][t] -= ey;
                any = true;
            }
        }
        if (!any) continue;
        float2* G1 = reinterpret_cast<float2*>(g1) + k * K;
        float2* G2 = reinterpret_cast<float2*>(g2) + k * K;
        for (int v = 0; v < n1; ++v) {
            float2 a = G1[v];
            a.x += gx[v][t];
            a.y += gy[v][t];
            G1[v] = a;
        }
        for (int v = 0; v < n2; ++v) {
            float2 a = G2[v];
            a.x += gx[n1 + v][t];
            a.y += gy[n1 + v][t];
            G2[v] = a;
        }
    }
}

unsigned var_grid(int64_t n) {
    int64_t b = (n + kVarThreads - 1) / kVarThreads;
    // one pair per thread up to 64 blocks per SM: measured faster than a
    // grid-stride loop over 16 blocks per SM (GIoU loss 229 -> 215 us per 1M pairs)
    const int64_t cap = (int64_t)sm_count() * 64;
    if (b > cap) b = cap;
    return (unsigned)(b < 1 ? 1 : b);
}

} // namespace

int64_t loss_var_partials(int64_t n) { return (int64_t)var_grid(n) * (kVarThreads / 32); }

dgal_status launch_loss_var_fwd(int variant, const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2,
                                int64_t n, int K, const float* weight, float scale, const float* u, float* ah,
                                uint64_t* aux, float* partials, cudaStream_t s) {
    const unsigned grid = var_grid(n);
    if (K == 4) {
        if (variant == 1) k_loss_var_fwd<4, 1><<<grid, kVarThreads, 0, s>>>(p1, c1, p2, c2, n, weight, scale, u, ah, aux, partials);
        else k_loss_var_fwd<4, 2><<<grid, kVarThreads, 0, s>>>(p1, c1, p2, c2, n, weight, scale, u, ah, aux, partials);
    } else {
        if (variant == 1) k_loss_var_fwd<8, 1><<<grid, kVarThreads, 0, s>>>(p1, c1, p2, c2, n, weight, scale, u, ah, aux, partials);
        else k_loss_var_fwd<8, 2><<<grid, kVarThreads, 0, s>>>(p1, c1, p2, c2, n, weight, scale, u, ah, aux, partials);
    }
    return check_launch("GIoU / DIoU forward");
}

dgal_status launch_loss_var_bwd(int variant, const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2,
                                int64_t n, int K, const float* weight, float scale, const float* dloss, const float* u,
                                const float* ah, const uint64_t* aux, float* g1, float* g2, cudaStream_t s) {
    const unsigned grid = var_grid(n);
    if (K == 4) {
        if (variant == 1)
            k_loss_var_bwd<4, 1><<<grid, kVarThreads, 0, s>>>(p1, c1, p2, c2, n, weight, scale, dloss, u, ah, aux, g1, g2);
        else
            k_loss_var_bwd<4, 2><<<grid, kVarThreads, 0, s>>>(p1, c1, p2, c2, n, weight, scale, dloss, u, ah, aux, g1, g2);
    } else {
        if (variant == 1)
            k_loss_var_bwd<8, 1><<<grid, kVarThreads, 0, s>>>(p1, c1, p2, c2, n, weight, scale, dloss, u, ah, aux, g1, g2);
        else
            k_loss_var_bwd<8, 2><<<grid, kVarThreads, 0, s>>>(p1, c1, p2, c2, n, weight, scale, dloss, u, ah, aux, g1, g2);
    }
    return check_launch("GIoU / DIoU backward");
}

} // namespace dgal
