/*
 * dgal.h — C ABI of libdgal, a GB300 (sm_103a) implementation of batched
 * convex-polygon intersection-over-union and its hand-written backward, after
 * DGAL ("Differentiable Computational Geometry for 2D and 3D machine
 * learning", arXiv:2011.11134).
 *
 * The calls follow the paper's `iou` / `iou_backward` listing (Sec. II-B):
 *   iou(p1, p2, nx, xflags)  = area(intersect(p1, p2)) / (area(p1) + area(p2)
 *                              - area(intersect(p1, p2))), recording nx (vertex
 *                              count of the intersection) and xflags (where each
 *                              intersection vertex comes from);
 *   iou_grad(p1, p2, grad, nx, xflags) -> (grad1, grad2), gradients shaped like
 *                              the polygons (Sec. III, last paragraph).
 * They are batched: `paired` (n independent pairs), `pairwise` (an N x M
 * matrix) and `pairwise_batched` (many ragged N_s x M_s matrices in one launch).
 *
 * Data layout (all device memory, caller-owned):
 *   polygons  float [n][K][2], x/y interleaved, convex, counter-clockwise
 *             (paper Sec. III: fixed-capacity point array, CCW), K in {4, 8};
 *             base pointer 16-byte aligned.
 *   counts    uint8 [n] vertex counts in [3, K], or NULL meaning "all K".
 *             Padded slots (index >= count) are ignored on input and receive
 *             zero gradient.
 *   iou       float [n] (paired) or [N][M] row-major (pairwise).
 *   nx        uint8 per pair / entry: intersection vertex count, 0 when the
 *             intersection has fewer than three vertices (then IoU = 0).
 *   xflags    uint8 [n][2K] (the paper's std::array<uint8_t, 8> for K = 4):
 *             code of each intersection vertex in counter-clockwise order,
 *             starting from the smallest code; unused slots are 0xFF.
 *               P1 vertex i                      -> i
 *               P2 vertex j                      -> 0x40 | j
 *               crossing of P1 edge i, P2 edge j -> 0x80 | (i << 3) | j
 *             (edge i joins vertex i to vertex i+1 mod count).
 *   degen     uint8 per pair, optional: bit 0 = near-degenerate pair (some
 *             |orientation| <= 1e-5 L^2, or a crossing within 1e-5 of an edge
 *             end, or nearly parallel crossing edges; L = largest |coordinate|
 *             relative to P1's vertex 0); bit 1 = FP64 orientation tests were
 *             used for this pair.
 *
 * Ownership and execution: the library never allocates on these paths and
 * never synchronises; every call enqueues kernels on `stream` (a
 * cudaStream_t; NULL = the legacy default stream) and returns.  n = 0 (or
 * N = 0 / M = 0 / S = 0) returns DGAL_OK without a launch.
 *
 * Errors: status codes only.  Arguments are validated on the host before any
 * launch (NULL required pointers, K not in {4, 8}, negative sizes, polygon or
 * output pointers not 16-byte aligned).  Problems only the device can see
 * (a count outside [3, K], a recorded nx or code out of range) set bits of a
 * per-device status word read by dgal_get_device_status(); kernels never trap.
 * dgal_last_error() returns a message for the last failing call on the calling
 * host thread.
 */
#ifndef DGAL_H
#define DGAL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    DGAL_OK = 0,
    DGAL_ERR_INVALID_ARG = 1,
    DGAL_ERR_UNSUPPORTED_K = 2,
    DGAL_ERR_ALIGNMENT = 3,
    DGAL_ERR_CUDA = 4,
    DGAL_ERR_WORKSPACE = 5,
    DGAL_ERR_DEVICE_STATUS = 6
} dgal_status;

/* Option bits for `flags`. */
#define DGAL_FP64_REFINE 0x1u /* near-degenerate pairs: orientation tests and crossing
                                 parameters in FP64 from the unrounded inputs */
#define DGAL_PLAIN 0x2u       /* the plain form: FP32 only, no refinement, one
                                 straightforward launch; the backward recomputes the clip */
#define DGAL_LOSS_GIOU 0x4u   /* dgal_iou_loss: the generalized IoU loss (see there) */
#define DGAL_LOSS_DIOU 0x8u   /* dgal_iou_loss: the distance IoU loss (see there) */
#define DGAL_VALIDATE 0x10u   /* debug: before its kernels, the call checks every input polygon
                                 for strict convexity and counter-clockwise order (the input
                                 contract, paper Sec. III) with dgal_validate_polygons'
                                 kernel; a polygon that fails sets DGAL_DEV_NOT_CONVEX, and
                                 the results for its pairs are undefined.  Applies to the
                                 device-memory paired, pairwise, 3D and loss calls; not to the
                                 ragged batch (its polygon counts live on the device) nor to the
                                 host-buffer call: check those arrays with
                                 dgal_validate_polygons.  Costs one extra pass over the polygons. */
#define DGAL_TEST_EXPIRE_WAIT 0x100u /* dgal_nms_rotated, for tests of the failure path: the
                                        greedy pass takes its wait-expiry path (DGAL_DEV_TIMEOUT,
                                        results incomplete) at its second block, once that block's
                                        copies have landed */

/* Device status bits (dgal_get_device_status). */
#define DGAL_DEV_BAD_COUNT 0x1u /* a vertex count outside [3, K] (pair treated as empty) */
#define DGAL_DEV_OVERFLOW 0x2u  /* more than 2K intersection candidates (pair treated as empty) */
#define DGAL_DEV_BAD_FLAGS 0x4u /* backward: nx > 2K or a code naming a missing vertex/edge */
#define DGAL_DEV_BAD_OFFSETS 0x8u /* ragged batch: offsets not starting at 0 or not N_s x M_s (scene skipped) */
#define DGAL_DEV_TIMEOUT 0x10u    /* a bounded wait on an asynchronous copy ran out (results incomplete) */
#define DGAL_DEV_NOT_CONVEX 0x20u /* DGAL_VALIDATE / dgal_validate_polygons: an input polygon is not strictly
                                     convex in counter-clockwise order */

/*
 * Paired IoU forward (paper Sec. II-B, `iou`): for k < n,
 *   iou[k] = A_i / (A_1 + A_2 - A_i) of p1[k], p2[k],
 * with nx[k], xflags[k][0..2K) and degen[k] recorded when the pointers are
 * non-NULL (nx and xflags must be both NULL or both set).
 * p1, p2: float [n][K][2]; c1, c2: uint8 [n] or NULL; iou: float [n] (required).
 */
dgal_status dgal_iou_paired(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                            int K, float* iou, uint8_t* nx, uint8_t* xflags, uint8_t* degen, uint32_t flags,
                            void* stream);

/*
 * Paired IoU backward (paper Sec. II-B, `iou_backward` / `iou_grad`): maps
 * grad_iou[k] = dL/dIoU onto both polygons' vertices through the recorded
 * intersection (nx, xflags).  grad_p1, grad_p2: float [n][K][2], overwritten
 * (padded slots set to 0).  When nx and xflags are both NULL (or DGAL_PLAIN is
 * set) the clip is recomputed from p1, p2 instead of read.
 */
dgal_status dgal_iou_backward(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                              int K, const float* grad_iou, const uint8_t* nx, const uint8_t* xflags,
                              float* grad_p1, float* grad_p2, uint32_t flags, void* stream);

/*
 * Forward + backward of paired IoU on HOST-resident data (a runtime
 * convenience; the paper has no counterpart): h_p1, h_p2 float [n][K][2],
 * h_c1, h_c2 uint8 [n] vertex counts or NULL (as for dgal_iou_paired),
 * h_grad float [n] = dL/dIoU in; h_iou float [n], h_g1, h_g2 float [n][K][2]
 * out (as dgal_iou_paired then dgal_iou_backward from the saved flags).
 * Results are bit-identical to the device-memory calls.  Two forms:
 *   direct: K = 4, all buffers (counts included) page-locked and mapped into the
 *     device's address space (cudaHostAlloc / pinned torch tensors; the
 *     polygon and gradient buffers 16-byte aligned): one kernel reads and
 *     writes the host buffers in place; `workspace` and `chunk` are not used
 *     (workspace may be NULL, chunk must still be positive);
 *   staged (otherwise): the pairs go through in chunks of `chunk` pairs over
 *     three staging slots of `workspace` (device memory, 256-byte aligned, at
 *     least dgal_iou_host_workspace_bytes(chunk, K) bytes, caller-owned):
 *     copies in, kernels and copies out of different chunks overlap on two
 *     copy streams of the library and the caller's stream.  The buffers
 *     should be pinned for the copies to overlap.  The copy streams and their
 *     events are created on the first staged call on a device (make it
 *     outside any stream capture) and reused, so staged calls from several
 *     host threads must be serialised by the caller.
 * The call is asynchronous and ordered on `stream`: the host buffers must
 * stay valid and unmodified until the stream reaches that point.
 */
size_t dgal_iou_host_workspace_bytes(int64_t chunk, int K);
dgal_status dgal_iou_fwd_bwd_host(const float* h_p1, const uint8_t* h_c1, const float* h_p2, const uint8_t* h_c2,
                                  const float* h_grad, int64_t n, int K, float* h_iou, float* h_g1, float* h_g2,
                                  void* workspace, size_t ws_bytes, int64_t chunk, uint32_t flags, void* stream);

/*
 * 3D IoU of paired boxes, each given as a bird's-eye-view polygon (as above)
 * and a vertical extent (the rotated 3D IoU loss use of the library, paper
 * Sec. IV-A):
 *   z1, z2   float [n][2] = (z_center, height), height > 0; 8-byte aligned.
 *   IoU3 = A_i ov / (A_1 h_1 + A_2 h_2 - A_i ov), ov = overlap of the two
 *   extents [z - h/2, z + h/2] (0 when disjoint); 0 when the union is not
 *   positive.  nx / xflags / degen record the bird's-eye-view intersection
 *   exactly as dgal_iou_paired does.
 */
dgal_status dgal_iou3d_paired(const float* p1, const uint8_t* c1, const float* z1, const float* p2, const uint8_t* c2,
                              const float* z2, int64_t n, int K, float* iou, uint8_t* nx, uint8_t* xflags,
                              uint8_t* degen, uint32_t flags, void* stream);

/*
 * Backward of dgal_iou3d_paired: grad_iou[k] = dL/dIoU3 -> grad_p1, grad_p2
 * (float [n][K][2]) and grad_z1, grad_z2 (float [n][2], dL/d(z_center,
 * height)), all overwritten.  At equal extent ends the subgradient of the
 * overlap takes P1's end.  nx / xflags: as for dgal_iou_backward.
 */
dgal_status dgal_iou3d_backward(const float* p1, const uint8_t* c1, const float* z1, const float* p2,
                                const uint8_t* c2, const float* z2, int64_t n, int K, const float* grad_iou,
                                const uint8_t* nx, const uint8_t* xflags, float* grad_p1, float* grad_z1,
                                float* grad_p2, float* grad_z2, uint32_t flags, void* stream);

/*
 * IoU loss with its gradient (the rotated-box IoU-loss use of the library,
 * paper Sec. IV-A):
 *   loss[0] = scale * sum_k w_k (1 - IoU(p1[k], p2[k]))      (w = NULL: all 1)
 *   grad_p1, grad_p2 = d loss / d p1, d p2  (float [n][K][2]; both NULL to skip)
 *   iou (float [n], optional) receives the IoUs.
 * With DGAL_LOSS_GIOU (the generalized IoU loss) each pair's term is instead
 *   w_k (1 - IoU_k + (A_h - U) / A_h),  A_h = area of the convex hull of both
 *   polygons' vertices, U = A_1 + A_2 - A_i the union;
 * with DGAL_LOSS_DIOU (the distance IoU loss)
 *   w_k (1 - IoU_k + rho2 / c2),  rho2 = squared distance between the two
 *   polygons' vertex means, c2 = squared diameter of that hull (the largest
 *   squared distance between two of the vertices).
 * The paper names the IoU loss; these two are its standard extensions.  A
 * pair whose union is not positive adds w_k and no gradient.
 * K = 4 or 8.  Runs the paired forward with the loss terms summed per warp and
 * the flags kept in `workspace`, then the paired backward with
 * dL/dIoU_k = -scale w_k formed in the kernel (for GIoU / DIoU a pass each way
 * adds the hull / centre terms); one block of the backward sums the per-warp
 * partials in a fixed order (a separate one-block launch does when no
 * gradient is wanted), so the loss is deterministic.  `workspace`: device
 * memory of at least dgal_iou_loss_workspace_bytes(n, K) bytes (0 for an
 * invalid K), 16-byte aligned, caller-owned; calls sharing it must not
 * overlap in time.  A call without gradients leaves in the workspace what
 * dgal_iou_loss_backward needs.  DGAL_PLAIN: FP32 only, and the backward
 * recomputes the clip.  DGAL_LOSS_GIOU and DGAL_LOSS_DIOU exclude each other.
 * n = 0 writes loss[0] = 0.
 */
size_t dgal_iou_loss_workspace_bytes(int64_t n, int K);
dgal_status dgal_iou_loss(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n, int K,
                          const float* weight, float scale, float* loss, float* iou, float* grad_p1, float* grad_p2,
                          void* workspace, size_t ws_bytes, uint32_t flags, void* stream);

/*
 * Backward of dgal_iou_loss for callers that take the loss's gradient later
 * (an autograd backward): after a dgal_iou_loss call with grad_p1 = grad_p2 =
 * NULL on the same inputs, weights, scale, flags and workspace, writes
 *   grad_p1, grad_p2 = dloss[0] * d loss / d p1, d p2   (float [n][K][2]),
 * with dloss a device pointer to one float (the upstream gradient of the
 * loss), read on the device, so nothing synchronises.  dloss = NULL means 1.
 * Same arguments and checks as dgal_iou_loss otherwise.
 */
dgal_status dgal_iou_loss_backward(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                                   int K, const float* weight, float scale, const float* dloss, float* grad_p1,
                                   float* grad_p2, void* workspace, size_t ws_bytes, uint32_t flags, void* stream);

/*
 * 3D IoU loss: dgal_iou_loss with the 3D IoU of dgal_iou3d_paired, i.e.
 * loss[0] = scale * sum_k w_k (1 - IoU3_k), its gradients grad_p1, grad_p2
 * (float [n][K][2]) and grad_z1, grad_z2 (float [n][2]); the four gradient
 * pointers are all NULL (loss only) or all set.  Same workspace as
 * dgal_iou_loss (dgal_iou_loss_workspace_bytes(n, K)).
 */
dgal_status dgal_iou3d_loss(const float* p1, const uint8_t* c1, const float* z1, const float* p2, const uint8_t* c2,
                            const float* z2, int64_t n, int K, const float* weight, float scale, float* loss,
                            float* iou, float* grad_p1, float* grad_z1, float* grad_p2, float* grad_z2,
                            void* workspace, size_t ws_bytes, uint32_t flags, void* stream);

/* Backward of dgal_iou3d_loss, as dgal_iou_loss_backward is of dgal_iou_loss
 * (the GIoU / DIoU flags are not taken by the 3D loss). */
dgal_status dgal_iou3d_loss_backward(const float* p1, const uint8_t* c1, const float* z1, const float* p2,
                                     const uint8_t* c2, const float* z2, int64_t n, int K, const float* weight,
                                     float scale, const float* dloss, float* grad_p1, float* grad_z1, float* grad_p2,
                                     float* grad_z2, void* workspace, size_t ws_bytes, uint32_t flags, void* stream);

/*
 * The intersection polygon of each pair (paper Sec. II-B, `intersect`, with
 * `area` of the result): verts float [n][2K][2] receives the nx[k]
 * intersection vertices in xflags order (counter-clockwise from the smallest
 * code; input vertices copied, crossings a + t (b - a) of the P1 edge, in
 * FP32), unused slots 0; area float [n] receives their shoelace area;
 * nx uint8 [n] and xflags uint8 [n][2K] as dgal_iou_paired (all required).
 * verts 16-byte aligned.  Runs the paired forward, then one vertex pass.
 */
dgal_status dgal_intersect_paired(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2, int64_t n,
                                  int K, float* verts, float* area, uint8_t* nx, uint8_t* xflags, uint32_t flags,
                                  void* stream);

/*
 * Area of each polygon (paper Sec. II-B, `area`): area[k] = shoelace area of
 * p[k] (float [n][K][2], CCW, counts c uint8 [n] or NULL); 0 and
 * DGAL_DEV_BAD_COUNT for a count outside [3, K].
 */
dgal_status dgal_area(const float* p, const uint8_t* c, int64_t n, int K, float* area, void* stream);

/*
 * Lines (paper Sec. III, "Lines": stored as the coefficients of their
 * equation, defined by two points in a differentiable manner).  A line is
 * float [3] = (a, b, c) with a x + b y + c = 0; points are float [2]
 * (8-byte aligned arrays).
 *   dgal_line_from_points: line[k] through p[k], q[k]:
 *     (a, b, c) = (p_y - q_y, q_x - p_x, p_x q_y - q_x p_y).
 *   dgal_line_from_points_backward: dL/d(a, b, c) [n][3] -> dL/dp, dL/dq
 *     [n][2] (overwritten).
 *   dgal_line_intersect: point[k] = (X / W, Y / W), X = b1 c2 - b2 c1,
 *     Y = c1 a2 - c2 a1, W = a1 b2 - a2 b1; parallel lines (W = 0) give
 *     non-finite coordinates.
 *   dgal_line_intersect_backward: dL/d(x, y) [n][2] -> dL/dl1, dL/dl2
 *     [n][3] (overwritten).
 */
dgal_status dgal_line_from_points(const float* p, const float* q, int64_t n, float* line, void* stream);
dgal_status dgal_line_from_points_backward(const float* p, const float* q, int64_t n, const float* grad_line,
                                           float* grad_p, float* grad_q, void* stream);
dgal_status dgal_line_intersect(const float* l1, const float* l2, int64_t n, float* point, void* stream);
dgal_status dgal_line_intersect_backward(const float* l1, const float* l2, int64_t n, const float* grad_point,
                                         float* grad_l1, float* grad_l2, void* stream);

/*
 * Forward and backward of the paired IoU in one call, for callers that know
 * dL/dIoU before the forward (a loss linear in the IoU, or a fixed upstream
 * gradient): the paper's `iou` and `iou_backward` (Sec. II-B) on the same
 * pairs.  Arguments as for dgal_iou_paired and dgal_iou_backward, all device
 * memory: grad_iou float [n] in, iou float [n] and grad_p1, grad_p2 float
 * [n][K][2] out (overwritten).
 *   K = 4: one kernel computes both halves, the clip state kept in registers
 *     between them (no flags are written; nx and xflags may be NULL).  The
 *     values are those of the two separate calls at one lane per pair (from
 *     the batch size where those calls take one lane per pair, see
 *     dgal_autotune class 1, they are bit-identical).
 *   K = 8: the forward and the backward kernels, with the flags in the
 *     caller's scratch nx uint8 [n], xflags uint8 [n][16] (16-byte aligned).
 * Errors as for dgal_iou_paired.
 */
dgal_status dgal_iou_fwd_bwd(const float* p1, const uint8_t* c1, const float* p2, const uint8_t* c2,
                             const float* grad_iou, int64_t n, int K, float* iou, float* grad_p1, float* grad_p2,
                             uint8_t* nx, uint8_t* xflags, uint32_t flags, void* stream);

/*
 * Pairwise IoU matrix: the paper's `iou` operation (Sec. II-B: intersect
 * the two convex polygons, take the shoelace areas, IoU = A_I / (A_1 + A_2 -
 * A_I)) applied to every one of the N x M pairs, as a rotated-box detector
 * does when it matches or suppresses boxes (Sec. IV):
 *   iou[i*M + j] = IoU(a[i], b[j]), nx[i*M + j] = vertex count of the
 *   intersection polygon (nx may be NULL).
 * a: float [N][K][2], b: float [M][K][2], CCW vertices (Sec. III), device,
 * 16-byte aligned; ca, cb: uint8 counts (3..K) or NULL for "all K"; iou: float
 * [N*M], nx: uint8 [N*M], device, caller-owned, overwritten.  N = 0 or M = 0
 * is a no-op returning DGAL_OK.  Invalid K, negative sizes or a NULL a / b /
 * iou return DGAL_ERR_INVALID_ARG, a misaligned pointer DGAL_ERR_ALIGNMENT, a
 * launch error DGAL_ERR_CUDA.
 * `flags`: DGAL_FP64_REFINE re-decides near-degenerate orientations in FP64.
 */
dgal_status dgal_iou_pairwise(const float* a, const uint8_t* ca, int64_t N, const float* b, const uint8_t* cb,
                              int64_t M, int K, float* iou, uint8_t* nx, uint32_t flags, void* stream);

/*
 * Ragged batch of S pairwise matrices in one persistent launch: the `iou`
 * operation of Sec. II-B over every pair of each scene, one scene per image
 * or point cloud of a detector's batch (Sec. IV), with scenes of different
 * sizes.  Scene s compares a[a_off[s] .. a_off[s+1]) with b[b_off[s] .. b_off[s+1]);
 * its N_s x M_s matrix is written row-major at iou + out_off[s] (and nx +
 * out_off[s]); out_off[s+1] - out_off[s] must equal N_s * M_s.
 * a_off, b_off, out_off: device int64 [S + 1], non-decreasing, a_off[0] =
 * b_off[0] = out_off[0] = 0 (read only on the device, so the call can be
 * captured in a CUDA graph).  workspace: device memory of at least
 * dgal_batched_workspace_bytes(S, K) bytes, 16-byte aligned, owned by the
 * caller; its contents on entry are ignored (the call re-initialises it).
 * Calls that share a workspace must not overlap in time.
 */
size_t dgal_batched_workspace_bytes(int S, int K);
dgal_status dgal_iou_pairwise_batched(int S, const int64_t* a_off, const int64_t* b_off, const int64_t* out_off,
                                      const float* a, const uint8_t* ca, const float* b, const uint8_t* cb, int K,
                                      float* iou, uint8_t* nx, void* workspace, size_t ws_bytes, uint32_t flags,
                                      void* stream);

/*
 * Allocation-free form of dgal_iou_pairwise_batched (the paper has no
 * counterpart; this is a convenience of this library).  For callers that
 * cannot allocate device memory when they call: code running while a stream
 * is captured into a CUDA graph, latency-critical loops where cudaMalloc would
 * stall the device, plugins whose host framework owns all device memory.
 * Arguments and results are those of dgal_iou_pairwise_batched without the
 * workspace: the scratch (queue counter and per-scene tile prefix) is one
 * fixed device array inside the library, about 33 KB, held by every GPU that
 * loads the library until the process exits.  At most 4096 scenes per call;
 * larger S returns DGAL_ERR_WORKSPACE.  No cudaMalloc or cudaFree is called.
 * The first call on a device looks up that array's device address once
 * (cudaGetSymbolAddress) with the device current; make that first call before
 * any stream capture.  All calls share the array and each call re-initialises
 * it, so calls whose kernels overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.
 */
dgal_status dgal_iou_pairwise_batched_noalloc(int S, const int64_t* a_off, const int64_t* b_off,
                                              const int64_t* out_off, const float* a, const uint8_t* ca,
                                              const float* b, const uint8_t* cb, int K, float* iou, uint8_t* nx,
                                              uint32_t flags, void* stream);

/*
 * The plain form of the ragged batch: one pairwise launch per scene with
 * host-side offsets (a_off_h, b_off_h, out_off_h are HOST int64 [S + 1]).
 */
dgal_status dgal_iou_pairwise_per_scene(int S, const int64_t* a_off_h, const int64_t* b_off_h,
                                        const int64_t* out_off_h, const float* a, const uint8_t* ca, const float* b,
                                        const uint8_t* cb, int K, float* iou, uint8_t* nx, uint32_t flags,
                                        void* stream);

/*
 * Rotated non-maximum suppression (greedy NMS over convex polygons, the use of
 * the pairwise IoU in rotated-box detection, paper Sec. IV): visit the boxes
 * by descending score, equal scores by lower index first, NaN scores last (as
 * -infinity); keep a box unless an already kept box overlaps it with
 * IoU > threshold.  The IoU is the FP32 IoU of dgal_iou_pairwise, so the
 * result equals that greedy rule applied to dgal_iou_pairwise's matrix.
 *   boxes    float [N][K][2] (16-byte aligned), counts uint8 [N] or NULL;
 *   scores   float [N];
 *   keep     int64 [N], receives the kept box indices in visiting order in
 *            keep[0 .. *num_keep); entries beyond are left unchanged;
 *   num_keep int64 [1] (device), receives the number of kept boxes;
 *   workspace: device memory of at least dgal_nms_workspace_bytes(N, K)
 *            bytes (about N^2 / 8 bytes for the suppression bitmap),
 *            16-byte aligned, caller-owned, contents ignored on entry; calls
 *            sharing it must not overlap in time.
 * N <= 131072 (larger N returns DGAL_ERR_INVALID_ARG and
 * dgal_nms_workspace_bytes returns 0).  N = 0 sets *num_keep = 0.
 * `flags`: DGAL_FP64_REFINE as for dgal_iou_pairwise.
 */
size_t dgal_nms_workspace_bytes(int64_t N, int K);
dgal_status dgal_nms_rotated(const float* boxes, const uint8_t* counts, const float* scores, int64_t N, int K,
                             float threshold, int64_t* keep, int64_t* num_keep, void* workspace, size_t ws_bytes,
                             uint32_t flags, void* stream);

/*
 * CUDA-graph form of dgal_iou_pairwise_batched: captures the call (with these
 * exact pointers and S) into an executable graph; dgal_graph_launch replays
 * it on `stream`.  Inputs may be rewritten in place between replays.
 * *graph receives an opaque handle; free it with dgal_graph_destroy.
 */
typedef struct dgal_graph_s* dgal_graph;
dgal_status dgal_batched_graph_create(dgal_graph* graph, int S, const int64_t* a_off, const int64_t* b_off,
                                      const int64_t* out_off, const float* a, const uint8_t* ca, const float* b,
                                      const uint8_t* cb, int K, float* iou, uint8_t* nx, void* workspace,
                                      size_t ws_bytes, uint32_t flags);
dgal_status dgal_graph_launch(dgal_graph graph, void* stream);
dgal_status dgal_graph_destroy(dgal_graph graph);

/*
 * Autotuner of the launch shapes, keeping the fastest per (device, K):
 *   config_class 0, the ragged batch: times candidate shapes (entries per
 *     tile, threads per block, resident blocks per SM) on a synthetic ragged
 *     problem generated on the current device;
 *   config_class 1, the paired calls: for quadrilaterals (K = 4), times one
 *     lane per pair against groups of 8 lanes per pair on the forward +
 *     backward of synthetic pairs at 2^10 .. 2^18 pairs, and sets the batch
 *     size below which groups are used (smaller batches are latency-bound;
 *     K = 8 pairs always take groups).  Untuned, that size is 1024.
 * cache_path (or, when NULL, the environment variable DGAL_TUNE_CACHE) names
 * a JSON file that is read first and rewritten with the result; NULL and no
 * variable means an in-memory cache only.  A cached ragged-batch shape
 * outside what the kernel accepts (threads a multiple of 32 up to 256, 1 to
 * 64 blocks per SM, a positive tile) is ignored and the shape tuned again.
 * This call allocates device memory and synchronises: call it before timing
 * or capturing, never inside a capture.
 */
dgal_status dgal_autotune(int K, int config_class, const char* cache_path);

/* The launch shape currently used by dgal_iou_pairwise_batched for K:
 * out[0] = entries per tile, out[1] = threads per block, out[2] = blocks per SM. */
dgal_status dgal_get_batched_config(int K, int32_t out[3]);

/* The launch shape currently used by the paired calls for K: *group_below =
 * the batch size (pairs) below which a group of 8 lanes takes each pair. */
dgal_status dgal_get_paired_config(int K, int64_t* group_below);

/*
 * Input check (the paper's convex, counter-clockwise polygons, Sec. III; the
 * library's results are undefined for other input): polygon k, its first
 * c[k] vertices (all K when c is NULL), passes when every vertex lies strictly
 * left of every edge it is not an end of, orient(v_i, v_i+1, v_m) > 0.  That
 * rejects clockwise order, reflex vertices, self-intersecting outlines and
 * repeated or collinear vertices.  Each test is decided in FP32 when its value
 * exceeds the FP32 error bound, else in FP64 from the raw inputs (exact sign).
 *   p    float [n][K][2], 16-byte aligned, device; c uint8 [n] or NULL;
 *   bad  uint8 [n] (device, nullable): 1 for a failing polygon, else 0;
 *   a failing polygon also sets DGAL_DEV_NOT_CONVEX in the device status word.
 * Counts outside [3, K] are not checked here (the IoU calls report them as
 * DGAL_DEV_BAD_COUNT; bad[k] = 0).  Asynchronous on `stream`.
 */
dgal_status dgal_validate_polygons(const float* p, const uint8_t* c, int64_t n, int K, uint8_t* bad, void* stream);

/* Reads (and, if clear != 0, resets) the current device's status word;
 * synchronises the device. */
dgal_status dgal_get_device_status(uint32_t* out, int clear);

/* Message of the last failing call on this host thread ("" if none). */
const char* dgal_last_error(void);

/* Library version: major * 10000 + minor * 100 + patch. */
int dgal_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DGAL_H */
