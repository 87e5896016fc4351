// The library's geometry operations exported on their own (paper Sec. II-B
// listing: intersect(p1, p2, xflags) returning the intersection polygon,
// area(polygon); Sec. III: lines stored as the coefficients of their
// equation and defined from two points differentiably).
//
//   dgal_intersect_paired  the paired forward (which records nx / xflags),
//                          then k_intersect_vertices: one thread per pair
//                          rebuilds the vertices named by the codes (input
//                          vertices copied, crossings as a_i + t ea_i in P1's
//                          local frame) and their shoelace area;
//   dgal_area              one thread per polygon, shoelace in the polygon's
//                          local frame (vertex 0 as origin);
//   dgal_line_*            elementwise, one thread per line / pair of lines,
//                          forward and hand-derived backward.
// All are HBM-bound streams: coalesced 8/16-byte loads and stores.
#include "dgal_geom.cuh"
#include "dgal_internal.h"

namespace dgal {

constexpr int kOpsThreads = 256;

static unsigned ops_grid(int64_t n) {
    int64_t b = (n + kOpsThreads - 1) / kOpsThreads;
    const int64_t cap = (int64_t)sm_count() * 32;
    return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

template <int K>
__global__ void __launch_bounds__(kOpsThreads)
k_intersect_vertices(const float* __restrict__ p1, const uint8_t* __restrict__ c1, const float* __restrict__ p2,
                     const uint8_t* __restrict__ c2, int64_t n, const uint8_t* __restrict__ nxs,
                     const uint8_t* __restrict__ xflags, float* __restrict__ verts, float* __restrict__ area,
                     uint32_t* status) {
    constexpr int C = 2 * K;
    uint32_t err = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        float px[K], py[K], qx[K], qy[K];
        load_poly<K>(p1 + k * 2 * K, px, py);
        load_poly<K>(p2 + k * 2 * K, qx, qy);
        const int n1 = c1 ? (int)c1[k] : K, n2 = c2 ? (int)c2[k] : K;
        uint32_t nx = nxs[k];
        const bool okc = n1 >= 3 && n1 <= K && n2 >= 3 && n2 <= K;
        if (nx > (uint32_t)C || !okc) {
            err |= okc ? kDevBadFlags : kDevBadCount;
            nx = 0;
        }
        const float ox = px[0], oy = py[0];
        float wx[C], wy[C];
        bool bad = false;
#pragma unroll
        for (int s = 0; s < C; ++s) {
            const uint32_t code = xflags[k * C + s];
            const uint32_t kind = code >> 6, i = (code >> 3) & 7u, j = code & 7u, v = code & 0x3Fu;
            float x = 0.f, y = 0.f;
            if ((uint32_t)s < nx) {
                if (kind == 0u) {
                    bad |= v >= (uint32_t)n1;
                    x = sel<K>(px, v);
                    y = sel<K>(py, v);
                } else if (kind == 1u) {
                    bad |= v >= (uint32_t)n2;
                    x = sel<K>(qx, v);
                    y = sel<K>(qy, v);
                } else if (kind == 2u && i < (uint32_t)n1 && j < (uint32_t)n2) {
                    const uint32_t i1 = (i + 1u < (uint32_t)n1) ? i + 1u : 0u;
                    const uint32_t j1 = (j + 1u < (uint32_t)n2) ? j + 1u : 0u;
                    const float ax = sel<K>(px, i) - ox, ay = sel<K>(py, i) - oy;
                    const float eax = (sel<K>(px, i1) - ox) - ax, eay = (sel<K>(py, i1) - oy) - ay;
                    const float bx = sel<K>(qx, j) - ox, by = sel<K>(qy, j) - oy;
                    const float ebx = (sel<K>(qx, j1) - ox) - bx, eby = (sel<K>(qy, j1) - oy) - by;
                    const float S = ebx * (ay - by) - eby * (ax - bx);
                    const float D = eax * eby - eay * ebx;
                    const float t = S / D;
                    x = ox + (ax + t * eax);
                    y = oy + (ay + t * eay);
                } else {
                    bad = true;
                }
            }
            wx[s] = x;
            wy[s] = y;
        }
        if (bad) {
            err |= kDevBadFlags;
            nx = 0;
#pragma unroll
            for (int s = 0; s < C; ++s) wx[s] = wy[s] = 0.f;
        }
        // shoelace of the rebuilt polygon about P1's vertex 0
        float two = 0.f;
#pragma unroll
        for (int s = 0; s < C; ++s) {
            // successor of slot s: slot s + 1, or slot 0 after the last vertex
            const bool last = (uint32_t)(s + 1) >= nx;
            const float xs = wx[s] - ox, ys = wy[s] - oy;
            const float xn = (last || s + 1 >= C) ? wx[0] - ox : wx[(s + 1) % C] - ox;
            const float yn = (last || s + 1 >= C) ? wy[0] - oy : wy[(s + 1) % C] - oy;
            two += ((uint32_t)s < nx) ? xs * yn - ys * xn : 0.f;
        }
        area[k] = nx >= 3u ? 0.5f * two : 0.f;
        float4* out = reinterpret_cast<float4*>(verts + k * 2 * C);
#pragma unroll
        for (int s = 0; s < C / 2; ++s) out[s] = make_float4(wx[2 * s], wy[2 * s], wx[2 * s + 1], wy[2 * s + 1]);
    }
    if (err) atomicOr(status, err);
}

template <int K>
__global__ void __launch_bounds__(kOpsThreads)
k_area(const float* __restrict__ p, const uint8_t* __restrict__ c, int64_t n, float* __restrict__ area,
       uint32_t* status) {
    uint32_t err = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        float x[K], y[K];
        load_poly<K>(p + k * 2 * K, x, y);
        const int m = c ? (int)c[k] : K;
        if (m < 3 || m > K) {
            err |= kDevBadCount;
            area[k] = 0.f;
            continue;
        }
        float s = 0.f;
#pragma unroll
        for (int v = 1; v + 1 < K; ++v) {
            // fan from vertex 0: triangles (0, v, v + 1) for v + 1 < m
            const float ux = x[v] - x[0], uy = y[v] - y[0], wx = x[v + 1] - x[0], wy = y[v + 1] - y[0];
            s += (v + 1 < m) ? ux * wy - uy * wx : 0.f;
        }
        area[k] = 0.5f * s;
    }
    if (err) atomicOr(status, err);
}

// Line through p and q: (a, b, c) = (p_y - q_y, q_x - p_x, p_x q_y - q_x p_y).
__global__ void __launch_bounds__(kOpsThreads)
k_line_from_points(const float2* __restrict__ p, const float2* __restrict__ q, int64_t n, float* __restrict__ line) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = __ldg(p + k), b = __ldg(q + k);
        line[3 * k] = a.y - b.y;
        line[3 * k + 1] = b.x - a.x;
        line[3 * k + 2] = a.x * b.y - b.x * a.y;
    }
}

__global__ void __launch_bounds__(kOpsThreads)
k_line_from_points_bwd(const float2* __restrict__ p, const float2* __restrict__ q, int64_t n,
                       const float* __restrict__ g, float2* __restrict__ gp, float2* __restrict__ gq) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float2 a = __ldg(p + k), b = __ldg(q + k);
        const float ga = g[3 * k], gb = g[3 * k + 1], gc = g[3 * k + 2];
        gp[k] = make_float2(gc * b.y - gb, ga - gc * b.x);
        gq[k] = make_float2(gb - gc * a.y, gc * a.x - ga);
    }
}

// Intersection of a1 x + b1 y + c1 = 0 and a2 x + b2 y + c2 = 0:
// (X / W, Y / W), X = b1 c2 - b2 c1, Y = c1 a2 - c2 a1, W = a1 b2 - a2 b1.
__global__ void __launch_bounds__(kOpsThreads)
k_line_intersect(const float* __restrict__ l1, const float* __restrict__ l2, int64_t n, float2* __restrict__ pt) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float a1 = l1[3 * k], b1 = l1[3 * k + 1], c1 = l1[3 * k + 2];
        const float a2 = l2[3 * k], b2 = l2[3 * k + 1], c2 = l2[3 * k + 2];
        const float W = a1 * b2 - a2 * b1;
        pt[k] = make_float2((b1 * c2 - b2 * c1) / W, (c1 * a2 - c2 * a1) / W);
    }
}

__global__ void __launch_bounds__(kOpsThreads)
k_line_intersect_bwd(const float* __restrict__ l1, const float* __restrict__ l2, int64_t n,
                     const float2* __restrict__ g, float* __restrict__ g1, float* __restrict__ g2) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float a1 = l1[3 * k], b1 = l1[3 * k + 1], c1 = l1[3 * k + 2];
        const float a2 = l2[3 * k], b2 = l2[3 * k + 1], c2 = l2[3 * k + 2];
        const float W = a1 * b2 - a2 * b1;
        const float x = (b1 * c2 - b2 * c1) / W, y = (c1 * a2 - c2 * a1) / W;
        const float2 gg = __ldg(g + k);
        const float gX = gg.x / W, gY = gg.y / W, gW = -(gg.x * x + gg.y * y) / W;
        g1[3 * k] = gW * b2 - gY * c2;
        g1[3 * k + 1] = gX * c2 - gW * a2;
        g1[3 * k + 2] = gY * a2 - gX * b2;
        g2[3 * k] = gY * c1 - gW * b1;
        g2[3 * k + 1] = gW * a1 - gX * c1;
        g2[3 * k + 2] = gX * b1 - gY * a1;
    }
}

// Input check of the DGAL_VALIDATE debug flag and dgal_validate_polygons:
// polygon k (its first n_k vertices) is a strictly convex polygon in
// counter-clockwise order exactly when every vertex lies strictly left of
// every edge it is not an end of, orient(v_i, v_i+1, v_m) > 0.  That also
// rejects clockwise order, reflex vertices, self-intersecting (star) outlines,
// repeated and collinear vertices.  Each test is taken in FP32 about v_i and
// trusted when its magnitude exceeds the FP32 error bound of the 2 x 2
// determinant of rounded differences, 8u (|ex dy| + |ey dx|); below that
// the FP64 value from the raw inputs decides (exact differences and products,
// so its sign is exact).  One thread per polygon, at most K (K - 2) tests; a
// count outside [3, K] is left to the other kernels (DGAL_DEV_BAD_COUNT).
template <int K>
__global__ void __launch_bounds__(kOpsThreads)
k_validate(const float* __restrict__ p, const uint8_t* __restrict__ c, int64_t n, uint8_t* __restrict__ bad,
           uint32_t* status) {
    uint32_t err = 0;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
        const float* pk = p + k * 2 * K;
        float x[K], y[K];
        load_poly<K>(pk, x, y);
        const int m = c ? (int)c[k] : K;
        bool ok = true;
        if (m >= 3 && m <= K) {
#pragma unroll
            for (int i = 0; i < K; ++i) {
                if (i >= m) break;
                const int i1 = (i + 1 < m) ? i + 1 : 0;
                const float ex = sel<K>(x, (uint32_t)i1) - x[i], ey = sel<K>(y, (uint32_t)i1) - y[i];
#pragma unroll
                for (int v = 0; v < K; ++v) {
                    if (v >= m || v == i || v == i1) continue;
                    const float dx = x[v] - x[i], dy = y[v] - y[i];
                    const float a = ex * dy, b = ey * dx;
                    const float o = a - b;
                    const float bound = 8.f * 5.9604645e-8f * (fabsf(a) + fabsf(b));
                    bool left = o > 0.f;
                    if (!(fabsf(o) > bound)) left = orient_raw(pk, i, i1, pk, v) > 0.0;
                    ok = ok && left;
                }
            }
        }
        if (bad) bad[k] = ok ? 0 : 1;
        if (!ok) err |= kDevNotConvex;
    }
    if (err) atomicOr(status, err);
}

dgal_status launch_validate(const float* p, const uint8_t* c, int64_t n, int K, uint8_t* bad, cudaStream_t s) {
    uint32_t* st = device_status_ptr();
    if (!st) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    if (n <= 0) return DGAL_OK;
    if (K == 4) k_validate<4><<<ops_grid(n), kOpsThreads, 0, s>>>(p, c, n, bad, st);
    else k_validate<8><<<ops_grid(n), kOpsThreads, 0, s>>>(p, c, n, bad, st);
    return check_launch("validate polygons");
}

} // namespace dgal

using namespace dgal;

namespace {

bool al(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

dgal_status need(const void* p, uintptr_t a, const char* name) {
    if (!p) return fail(DGAL_ERR_INVALID_ARG, "%s is NULL", name);
    if (!al(p, a)) return fail(DGAL_ERR_ALIGNMENT, "%s is not %d-byte aligned", name, (int)a);
    return DGAL_OK;
}

#define OPS_TRY(expr)                   \
    do {                                \
        dgal_status _st = (expr);       \
        if (_st != DGAL_OK) return _st; \
    } while (0)

} // namespace

extern "C" {

dgal_status dgal_intersect_paired(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                                  int K, float* verts, float* area, uint8_t* nx, uint8_t* xflags, uint32_t flags,
                                  void* stream) {
    if (K != 4 && K != 8) return fail(DGAL_ERR_UNSUPPORTED_K, "K = %d is not supported (K must be 4 or 8)", K);
    if (n < 0) return fail(DGAL_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    if (n == 0) return DGAL_OK;
    OPS_TRY(need(p1, 16, "p1"));
    OPS_TRY(need(p2, 16, "p2"));
    OPS_TRY(need(verts, 16, "verts"));
    OPS_TRY(need(area, 4, "area"));
    OPS_TRY(need(nx, 1, "nx"));
    OPS_TRY(need(xflags, K == 4 ? 8 : 16, "xflags"));
    if (!device_status_ptr()) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    cudaStream_t s = (cudaStream_t)stream;
    // the forward writes its IoU into `area`; the vertex pass overwrites it
    OPS_TRY(launch_paired_fwd(p1, c1, p2, c2, n, K, area, nx, xflags, nullptr, flags, s));
    if (K == 4)
        k_intersect_vertices<4><<<ops_grid(n), kOpsThreads, 0, s>>>(p1, c1, p2, c2, n, nx, xflags, verts, area,
                                                                   device_status_ptr());
    else
        k_intersect_vertices<8><<<ops_grid(n), kOpsThreads, 0, s>>>(p1, c1, p2, c2, n, nx, xflags, verts, area,
                                                                   device_status_ptr());
    return check_launch("intersect vertices");
}

dgal_status dgal_area(const float* p, const uint8_t* c, int64_t n, int K, float* area, void* stream) {
    if (K != 4 && K != 8) return fail(DGAL_ERR_UNSUPPORTED_K, "K = %d is not supported (K must be 4 or 8)", K);
    if (n < 0) return fail(DGAL_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    if (n == 0) return DGAL_OK;
    OPS_TRY(need(p, 16, "p"));
    OPS_TRY(need(area, 4, "area"));
    if (!device_status_ptr()) return fail(DGAL_ERR_CUDA, "device status word unavailable");
    cudaStream_t s = (cudaStream_t)stream;
    if (K == 4) k_area<4><<<ops_grid(n), kOpsThreads, 0, s>>>(p, c, n, area, device_status_ptr());
    else k_area<8><<<ops_grid(n), kOpsThreads, 0, s>>>(p, c, n, area, device_status_ptr());
    return check_launch("area");
}

dgal_status dgal_line_from_points(const float* p, const float* q, int64_t n, float* line, void* stream) {
    if (n < 0) return fail(DGAL_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    if (n == 0) return DGAL_OK;
    OPS_TRY(need(p, 8, "p"));
    OPS_TRY(need(q, 8, "q"));
    OPS_TRY(need(line, 4, "line"));
    k_line_from_points<<<ops_grid(n), kOpsThreads, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float2*>(p), reinterpret_cast<const float2*>(q), n, line);
    return check_launch("line from points");
}

dgal_status dgal_line_from_points_backward(const float* p, const float* q, int64_t n, const float* grad_line,
                                           float* grad_p, float* grad_q, void* stream) {
    if (n < 0) return fail(DGAL_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    if (n == 0) return DGAL_OK;
    OPS_TRY(need(p, 8, "p"));
    OPS_TRY(need(q, 8, "q"));
    OPS_TRY(need(grad_line, 4, "grad_line"));
    OPS_TRY(need(grad_p, 8, "grad_p"));
    OPS_TRY(need(grad_q, 8, "grad_q"));
    k_line_from_points_bwd<<<ops_grid(n), kOpsThreads, 0, (cudaStream_t)stream>>>(
        reinterpret_cast<const float2*>(p), reinterpret_cast<const float2*>(q), n, grad_line,
        reinterpret_cast<float2*>(grad_p), reinterpret_cast<float2*>(grad_q));
    return check_launch("line from points backward");
}

dgal_status dgal_line_intersect(const float* l1, const float* l2, int64_t n, float* point, void* stream) {
    if (n < 0) return fail(DGAL_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    if (n == 0) return DGAL_OK;
    OPS_TRY(need(l1, 4, "l1"));
    OPS_TRY(need(l2, 4, "l2"));
    OPS_TRY(need(point, 8, "point"));
    k_line_intersect<<<ops_grid(n), kOpsThreads, 0, (cudaStream_t)stream>>>(l1, l2, n,
                                                                            reinterpret_cast<float2*>(point));
    return check_launch("line intersect");
}

dgal_status dgal_line_intersect_backward(const float* l1, const float* l2, int64_t n, const float* grad_point,
                                         float* grad_l1, float* grad_l2, void* stream) {
    if (n < 0) return fail(DGAL_ERR_INVALID_ARG, "n = %lld is negative", (long long)n);
    if (n == 0) return DGAL_OK;
    OPS_TRY(need(l1, 4, "l1"));
    OPS_TRY(need(l2, 4, "l2"));
    OPS_TRY(need(grad_point, 8, "grad_point"));
    OPS_TRY(need(grad_l1, 4, "grad_l1"));
    OPS_TRY(need(grad_l2, 4, "grad_l2"));
    k_line_intersect_bwd<<<ops_grid(n), kOpsThreads, 0, (cudaStream_t)stream>>>(
        l1, l2, n, reinterpret_cast<const float2*>(grad_point), grad_l1, grad_l2);
    return check_launch("line intersect backward");
}

} // extern "C"
