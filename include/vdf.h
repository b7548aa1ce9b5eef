/*
 * vdf.h -- C ABI of the GB300 directional vector filter library (libvdf.so).
 *
 * The library implements the order-statistics directional filters of
 * M. E. Celebi, "Real-time implementation of order-statistics based
 * directional filters":
 *   - Section II: each pixel of an M x N RGB image is replaced by one member
 *     of the sqrt(n) x sqrt(n) window centred on it (n = win * win), the
 *     member that minimises an aggregated distance to all n members.
 *   - BVDF, Eq. (2): aggregated angle  sum_j A(x_i, x_j),
 *     A(x, y) = acos(<x,y> / (|x| |y|)).
 *   - DDF, Eq. (3): (sum_j A)^p * (sum_j L2)^(1-p), L2 the Minkowski distance
 *     of Eq. (1) at order 2; p = 1/2 orders like Eq. (3)'s plain product.
 *   - VMF, Eq. (1): aggregated Minkowski distance sum_j L(x_i, x_j),
 *     L(x, y) = (sum_k |x_k - y_k|^o)^(1/o).  vdf_filter_lp selects the order
 *     o in {1, 2} or the limit of infinite order (max_k |x_k - y_k|) for the
 *     VMF and for the distance term of the DDF; every other entry point uses
 *     order 2.
 *   - Method 1 (Section 2.1, Eqs. (4)-(6), Table 1): A replaced by a degree-q
 *     minimax polynomial.  Method 2 (Section 2.2, Eq. (7)): A replaced by the
 *     chromaticity distance B; inside DDF B goes through Eq. (10) first.
 *
 * Conventions fixed by this library (the paper is silent):
 *   - window members in raster order, index i = (dy+R)*win + (dx+R), centre
 *     (n-1)/2; pixels outside the image are replaced by the nearest edge pixel;
 *   - a zero vector is at angle pi/2 from every vector (cosine taken as 0) and
 *     has chromaticity 0;
 *   - DDF uses max(sum_j A, 0) inside the power and 0^0 = 1;
 *   - ties: the centre if it attains the minimum, else the lowest index.
 *
 * Images are uint8, HWC (row-major, 3 bytes per pixel, row pitch 3*N bytes)
 * unless stated.  Device pointers must come from the same CUDA context as
 * the stream.  Every call is asynchronous on `stream` (a cudaStream_t, NULL
 * for the legacy default stream) unless stated otherwise.  The library never
 * allocates device memory inside these calls: scratch space is passed in as
 * a caller-owned `workspace`.  Calls return VDF_OK (0) or a negative
 * vdf_status; nothing throws or aborts across the ABI.
 */
#ifndef VDF_H
#define VDF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { VDF_BVDF = 0, VDF_DDF = 1, VDF_VMF = 2 } vdf_filter_kind;

/* Minkowski order argument of vdf_filter_lp for the limit of infinite order. */
#define VDF_MINKOWSKI_INF 0

/* Distance used in place of A (Section II; Methods 1 and 2). */
typedef enum { VDF_DIST_EXACT = 0, VDF_DIST_MINIMAX = 1, VDF_DIST_RGB = 2 } vdf_dist_mode;

/* VDF_PREC_FP64: every pair term, aggregate and comparison in double
 * precision; ties are aggregates within 1e-11 (relative, floor 1e-3) of the
 * minimum (in the log domain for DDF).
 * VDF_PREC_FP32_RECHECK: single precision with a per-candidate certified
 * error bound; a pixel whose minimum is not separated by the bounds, and
 * whose near-minimal members are not provably equal (identical vectors, or
 * collinear ones for BVDF, or exact zeros), is recomputed by the FP64 path.
 * Both precisions therefore select the same member on every pixel. */
typedef enum { VDF_PREC_FP64 = 0, VDF_PREC_FP32_RECHECK = 1 } vdf_precision;

typedef enum {
    VDF_OK = 0,
    VDF_E_INVALID = -1,     /* null pointer, bad size, bad win / p / q, aliasing */
    VDF_E_CUDA = -2,        /* a CUDA launch or copy failed (see vdf_last_cuda_error) */
    VDF_E_OVERFLOW = -3,    /* reserved, never returned: the recheck list has an
                               entry for every pixel, so it cannot overflow */
    VDF_E_TIMEOUT = -4,     /* reserved, never returned: no kernel of this
                               library waits on the device */
    VDF_E_WORKSPACE = -5,   /* workspace missing or smaller than required */
    VDF_E_UNSUPPORTED = -6  /* valid request the library does not implement */
} vdf_status;

/* Human-readable text of a status code (static storage). */
const char *vdf_strerror(int status);

/* Text of the last CUDA error seen by this thread (static storage). */
const char *vdf_last_cuda_error(void);

/* Bytes of device workspace vdf_filter needs for an M x N image with the
 * given precision (0 for VDF_PREC_FP64).  Returns 0 on invalid sizes. */
size_t vdf_workspace_bytes(int M, int N, int precision);

/*
 * Filter one M x N uint8 HWC image on the device.
 *   img        device, M*N*3 bytes.  Not modified.
 *   out        device, M*N*3 bytes: the selected member's RGB.  Must not
 *              overlap img.
 *   index_out  device, M*N int8 (may be NULL): selected raster index 0..n-1.
 *   agg_out    device, M*N*n*2 doubles (may be NULL; FP64 precision only):
 *              per pixel and member i, sum_j A_ij then sum_j L2_ij (the
 *              latter 0 for BVDF).  For Method 2 in DDF the first value is
 *              1.436437 * sum_j B_ij + 0.027664 * n (Eq. (10)).
 *   win        3, 5 or 7 (Section II's sqrt(n) x sqrt(n) window; n = 49
 *              still fits the int8 index).  3 and 5 run the tile kernels,
 *              which compute each pair term once for all windows sharing
 *              it; 7 runs a kernel with one warp per output pixel (every
 *              member's aggregate formed over its window directly; in FP64
 *              each unordered pair once per window).
 *              filter: vdf_filter_kind (VDF_VMF at order 2).
 *              p: DDF exponent, [0, 1].
 *   dist_mode  vdf_dist_mode (ignored for VDF_VMF).  minimax_q: 2, 3 or 4
 *              (used for MINIMAX only).
 *   precision  vdf_precision.
 *   workspace  device, vdf_workspace_bytes(M, N, precision) bytes, 256-byte
 *              aligned (NULL allowed when that size is 0).  Its contents on
 *              return are the recheck counters (see vdf_workspace_stats).
 * Errors: VDF_E_INVALID, VDF_E_WORKSPACE, VDF_E_UNSUPPORTED, VDF_E_CUDA.
 */
int vdf_filter(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode, int minimax_q,
               int precision, uint8_t *out, int8_t *index_out, double *agg_out, void *workspace,
               size_t workspace_bytes, void *stream);

/*
 * vdf_filter with the Minkowski order of the distance term of Eq. (1):
 *   minkowski_order  1, 2, or VDF_MINKOWSKI_INF.  Used by VDF_VMF and
 *              VDF_DDF (ignored for VDF_BVDF).
 * VDF_VMF: p and dist_mode are ignored (the filter has no angular term); at
 * orders 1 and infinity its aggregates are exact integers in both precisions
 * and no pixel is rechecked.  VDF_DDF at order 1 or infinity needs
 * VDF_DIST_EXACT (else VDF_E_UNSUPPORTED).  agg_out, when given, holds
 * sum_j A (0 for the VMF) then sum_j L per member.  Other arguments and
 * errors as for vdf_filter (VDF_E_INVALID for any other order).
 */
int vdf_filter_lp(const uint8_t *img, int M, int N, int win, int filter, double p, int minkowski_order,
                  int dist_mode, int minimax_q, int precision, uint8_t *out, int8_t *index_out, double *agg_out,
                  void *workspace, size_t workspace_bytes, void *stream);

/*
 * ACWDDF, Eq. (9) (Section 3.2): per pixel, the DDF output (Eq. (3), plain
 * product, A of dist_mode; Method 2 through Eq. (10)) if
 *     sum_{k=lambda}^{lambda+2} A(y_k, x_d) * L2(y_k, x_d) > T,
 * else the centre x_d, where y_k is the centre-weighted VMF output at
 * smoothing level k: argmin_i sum_j w_j(k) L2(x_i, x_j), w_d(k) = n - 2k + 2,
 * w_j = 1 otherwise.  Readings: Eq. (9) names the outputs of the test CWDDF^k
 * but defines CWVMF^k, which are used; the test is strict.  The paper sets
 * lambda = 2 and T = 10.8.
 *   win        3 or 5 (VDF_E_UNSUPPORTED for 7).
 *   lambda     1 .. d - 2 with d = (win*win + 1)/2 (so every level k <= d).
 *   T          finite threshold.
 * Other arguments as vdf_filter (filter fixed to the DDF, p = 1/2).  With
 * VDF_PREC_FP32_RECHECK the DDF choice, each CWVMF level and the switch are
 * decided in FP32 with certified bounds; a pixel where any of them is open is
 * recomputed entirely by the FP64 path, so both precisions give the same
 * result.  Errors: VDF_E_INVALID (also for lambda or T out of range),
 * VDF_E_WORKSPACE, VDF_E_CUDA.
 */
int vdf_filter_acwddf(const uint8_t *img, int M, int N, int win, int dist_mode, int minimax_q, int lambda, double T,
                      int precision, uint8_t *out, int8_t *index_out, void *workspace, size_t workspace_bytes,
                      void *stream);

/*
 * The two stages of vdf_filter with VDF_PREC_FP32_RECHECK, for callers that
 * want to time or overlap them separately.  vdf_fp32_pass zeroes the recheck
 * counters, runs the FP32 tile kernel (writing out / index_out for every
 * pixel, provisional where the bounds do not separate the minimum) and
 * appends those pixels to the list in `workspace`.  vdf_fp64_recheck then
 * recomputes the listed pixels with the FP64 path (it reads the list length
 * on the device; no host synchronisation).  Arguments as for vdf_filter.
 */
int vdf_fp32_pass(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode, int minimax_q,
                  uint8_t *out, int8_t *index_out, void *workspace, size_t workspace_bytes, void *stream);
int vdf_fp64_recheck(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode,
                     int minimax_q, uint8_t *out, int8_t *index_out, void *workspace, size_t workspace_bytes,
                     void *stream);

/* Recheck counters of the last vdf_filter that used `workspace`: pixels
 * re-evaluated in FP64 and a non-zero overflow flag.  Synchronises `stream`
 * and copies 8 bytes to the host. */
int vdf_workspace_stats(const void *workspace, int64_t *rechecked, int32_t *overflow, void *stream);

/*
 * Counters of the last FP32 call (vdf_filter / vdf_fp32_pass / vdf_filter_lp /
 * vdf_filter_acwddf / vdf_filter_f32 with VDF_PREC_FP32_RECHECK, or
 * vdf_filter_batch) that used `workspace`:
 *   rechecked        pixels listed for the FP64 recheck (their near-minimal
 *                    members were not separated by the certified bounds);
 *   structural_ties  pixels with several near-minimal members that the FP32
 *                    path proved equal (identical vectors; collinear ones for
 *                    BVDF; exact zeros; equal integer scores of the VMF at
 *                    orders 1 and infinity), decided by the tie rule without
 *                    a recheck (Section II defines the selection as an
 *                    argmin; the tie rule is this library's);
 *   overflow         always 0 (the list has an entry per pixel).
 * Synchronises `stream` and copies 256 bytes to the host.  Errors:
 * VDF_E_INVALID for a null pointer, VDF_E_CUDA.
 */
typedef struct {
    int64_t rechecked;
    int64_t structural_ties;
    int32_t overflow;
} vdf_stats;
int vdf_read_stats(const void *workspace, vdf_stats *stats, void *stream);

/*
 * Same as vdf_filter with host buffers: copies img (M*N*3 bytes, host) to
 * the device, filters, copies out (M*N*3) and index_out (M*N, may be NULL)
 * back, and waits for the stream.  dev_buffer is device scratch of
 * vdf_host_buffer_bytes(M, N, precision) bytes holding the device copies and
 * the workspace.  Host buffers should be pinned for full copy speed.
 */
size_t vdf_host_buffer_bytes(int M, int N, int precision);
int vdf_filter_host(const uint8_t *img_host, int M, int N, int win, int filter, double p, int dist_mode,
                    int minimax_q, int precision, uint8_t *out_host, int8_t *index_out_host, void *dev_buffer,
                    size_t dev_buffer_bytes, void *stream);

/*
 * A sequence of count host frames of equal size through vdf_filter, the
 * copies of each frame overlapping the filtering of its neighbours (frames
 * of a video; the paper filters one image at a time and has no such call).
 * Three device slots of vdf_host_buffer_bytes(M, N, precision) bytes
 * (rounded up to 256) are used in turn; library-owned streams (four per
 * device, created on first use) carry the upload, the FP32 pass (or the FP64
 * filter), the FP64 recheck and the download, ordered by events, so the
 * upload of frame i + 1 and the download of frame i - 1 run while frame i is
 * filtered, and the recheck of frame i beside the next passes.
 *   img_host[i]        host, M*N*3 uint8 (HWC); pinned for overlap
 *   out_host[i]        host, M*N*3 uint8
 *   index_out_host     NULL, or an array whose entries are NULL or host M*N int8
 *   dev_buffer         device, 256-byte aligned, vdf_host_frames_buffer_bytes(M, N,
 *                      precision) bytes, owned by the caller
 *   stream             the work starts after the work queued on it, and it waits
 *                      for the last download; the call returns when every frame
 *                      is on the host (also after an error)
 * Errors: VDF_E_INVALID for bad sizes or null frame pointers (count = 0 is
 * a no-op); VDF_E_WORKSPACE for a short or misaligned buffer; the filter's
 * own errors (its argument checks run on the first frame); VDF_E_CUDA.
 * Calls on one device are serialised by a lock.
 */
size_t vdf_host_frames_buffer_bytes(int M, int N, int precision);
int vdf_filter_host_frames(const uint8_t *const *img_host, uint8_t *const *out_host, int8_t *const *index_out_host,
                           int count, int M, int N, int win, int filter, double p, int dist_mode, int minimax_q,
                           int precision, void *dev_buffer, size_t dev_buffer_bytes, void *stream);

/*
 * Float32 batch variant (the differentiable path).  img: device, B x 3 x M x N
 * float32 (NCHW, any non-negative values, e.g. RGB in [0, 1]); out: same
 * shape; index_out: device, B x M x N int8 (may be NULL, but the backward
 * pass needs it).  Only VDF_BVDF and VDF_DDF with VDF_DIST_EXACT are
 * supported for float input, at windows 3 and 5 (else VDF_E_UNSUPPORTED).  The
 * FP64 precision computes the pair terms from the float32 values exactly
 * promoted to double.  VDF_PREC_FP32_RECHECK computes them in FP32 on
 * exponent-normalised pixels with certified bounds (Kahan cross products)
 * and rechecks in FP64 the pixels the bounds leave open, the windows with an
 * aggregate below 2^-23, and every tile holding a negative, non-finite,
 * subnormal or extreme component; it selects what the FP64 precision
 * selects.  It needs workspace of vdf_workspace_bytes(B * M, N, precision)
 * bytes (256-byte aligned).  Errors as vdf_filter.
 */
int vdf_filter_f32(const float *img, int B, int M, int N, int win, int filter, double p, int dist_mode,
                   int minimax_q, int precision, float *out, int8_t *index_out, void *workspace,
                   size_t workspace_bytes, void *stream);

/*
 * Gradient of vdf_filter_f32 with respect to its input, given the saved
 * index map: the forward pass copies x(src(p)) to y(p), src(p) = the selected
 * member (clamped to the image), so grad_x(q) = sum of grad_y(p) over all p
 * with src(p) = q.  Computed as a gather over each q's window-sized
 * neighbourhood in a fixed order (deterministic, no atomics).
 *   grad_y, grad_x: device, B x 3 x M x N float32 (must not overlap);
 *   index: device, B x M x N int8 from vdf_filter_f32 with the same win.
 *          A byte outside 0 .. win*win - 1 (e.g. from a map made with a
 *          different window) selects no source: its pixel passes no gradient.
 * There is no counterpart in the paper (it does not differentiate the
 * filters); this is the exact gradient of the selection away from ties.
 */
/* win: 3 or 5. */
int vdf_backward_f32(const float *grad_y, const int8_t *index, int B, int M, int N, int win, float *grad_x,
                     void *stream);

/*
 * vdf_filter with VDF_PREC_FP32_RECHECK for callers that cannot allocate
 * device memory (where cudaMalloc is forbidden after start-up, such as
 * real-time loops that must not block on the allocator, or hosts that own all
 * device memory and pass in only the image buffers).  It takes no workspace:
 * the recheck counters and list live in a fixed device array inside the
 * library (256 bytes + 16 MiB, held on every GPU that loads the library until
 * the process exits).  The paper has no counterpart; this is an interface
 * convenience.
 *   - M * N must not exceed 2,097,152 pixels (2^21, e.g. 1920 x 1080);
 *     larger images return VDF_E_WORKSPACE and launch nothing.
 *   - The first call on a device looks up the array's device address (which
 *     may load the library's device code): make it before any stream capture.
 *     The address is kept for the process; after cudaDeviceReset on a
 *     device, do not call this function on that device again.
 *   - Arguments are checked as by vdf_filter (VDF_E_INVALID) before the size
 *     limit (VDF_E_WORKSPACE).
 *   - All calls share the array: calls that overlap on the GPU race and must
 *     be serialised by the caller.
 * Other arguments, results and errors as vdf_filter.
 */
int vdf_filter_noalloc(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode,
                       int minimax_q, uint8_t *out, int8_t *index_out, void *stream);

/*
 * Tile-shape autotuner of the FP32 kernel.  The kernel exists in
 * vdf_num_tile_shapes() output-tile shapes (vdf_tile_shape gives width x
 * height).  vdf_autotune times every shape on the given image with the given
 * configuration (`reps` timed launches each after one warm-up, CUDA events
 * on `stream`; the call waits for the stream), records the fastest for
 * (win, filter, dist_mode) in a process-wide table used by vdf_filter,
 * (windows 3 and 5: the 7x7 kernel has no tile shapes, VDF_E_UNSUPPORTED)
 * vdf_fp32_pass and vdf_plan_create, and returns it in *best_shape and its
 * mean time in *best_ms.  Buffers and workspace as for vdf_fp32_pass (the
 * image is filtered; out / index_out receive valid results).
 * vdf_get_tuned_shape / vdf_set_tuned_shape read or restore table entries
 * (for example from a cache file).  The paper has no counterpart.
 * The DDF 5x5 at p = 1/4, 1/2 or 3/4 with the exact or chromaticity terms
 * runs kernels of its own (score slots: each (window, member) slot holds the
 * score, so smaller tiles fit two blocks per SM) and has table entries of its
 * own for each of the three exponents: vdf_autotune at such a p records into
 * that p's entry, vdf_get_tuned_shape_p(..., p) reads the entry used at
 * exponent p, vdf_get_tuned_shape reads the entry of the other exponents, and
 * vdf_set_tuned_shape sets them all.
 * vdf_autotune_acwddf does the same for the ACWDDF (its arguments as
 * vdf_filter_acwddf, with the FP32 precision): it times the ACWDDF kernel in
 * every shape and records the fastest in an entry of its own, which
 * vdf_filter_acwddf reads (vdf_set_tuned_shape with filter VDF_DDF sets it
 * too).  Window 7: VDF_E_UNSUPPORTED.
 */
int vdf_num_tile_shapes(void);
int vdf_tile_shape(int shape, int *tile_w, int *tile_h);
int vdf_autotune(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode, int minimax_q,
                 uint8_t *out, int8_t *index_out, void *workspace, size_t workspace_bytes, int reps, void *stream,
                 int *best_shape, float *best_ms);
int vdf_autotune_acwddf(const uint8_t *img, int M, int N, int win, int dist_mode, int minimax_q, int lambda,
                        double T, uint8_t *out, int8_t *index_out, void *workspace, size_t workspace_bytes, int reps,
                        void *stream, int *best_shape, float *best_ms);
int vdf_get_tuned_shape(int win, int filter, int dist_mode);
int vdf_get_tuned_shape_p(int win, int filter, int dist_mode, double p);
int vdf_set_tuned_shape(int win, int filter, int dist_mode, int shape);

/*
 * Batches of uneven images (FP32 certified path).  Each image has its own
 * size, window (3 or 5), filter and DDF exponent; the distance mode (exact,
 * Method 1 with degree minimax_q, or Method 2) is one per plan
 * (vdf_plan_create: VDF_E_INVALID for another mode or, with Method 1, a q
 * outside 2..4).  A plan holds, on the host, one descriptor per image with
 * the tile shape the autotuner table gives its configuration, and the tile
 * and pixel offsets of the batch.
 *   vdf_plan_create      validates the descriptors (the plan keeps a copy;
 *                        device pointers must stay valid while it is used).
 *   vdf_plan_workspace_bytes  device workspace: counters, descriptors, the
 *                        image index of every work item (4 bytes per tile) and
 *                        a recheck list entry per pixel of the batch.
 *   vdf_plan_upload      copies the descriptors and the item table into
 *                        `workspace` (once per workspace, before
 *                        vdf_filter_batch or a capture).
 *   vdf_filter_batch     zeroes the counters, launches one tile kernel per
 *                        configuration present (window, filter, tuned tile
 *                        shape; each at its own block size and occupancy) over
 *                        that configuration's (image, tile) work items, then
 *                        one persistent FP64 recheck kernel.  Stream-ordered,
 *                        no host sync, no allocation: it can be captured in a
 *                        CUDA graph.
 *   vdf_plan_set_persistent  selects the form of the tile kernels: 0 (the
 *                        default) one CTA per work item, its image read from a
 *                        per-item table in the workspace; 1 persistent, as
 *                        many CTAs as fit on the SMs, each taking work items
 *                        from an atomic counter.  Same results; the per-item
 *                        form is the faster one (the persistent loop costs
 *                        registers).  Drops a graph captured for the other
 *                        form.
 *   vdf_plan_graph_launch  captures vdf_filter_batch into a CUDA graph on the
 *                        first call for a given workspace, then launches the
 *                        graph on `stream`.
 *   vdf_plan_destroy     frees the plan and its graph.
 * Recheck counters are read with vdf_workspace_stats(workspace, ...).
 */
typedef struct {
    const uint8_t *img;  /* device, M*N*3 */
    uint8_t *out;        /* device, M*N*3, must not overlap img */
    int8_t *index_out;   /* device, M*N, or NULL */
    int M, N;
    int win;             /* 3 or 5 */
    int filter;          /* vdf_filter_kind */
    double p;            /* DDF exponent in [0, 1] */
} vdf_image_desc;

typedef struct vdf_plan vdf_plan;

int vdf_plan_create(vdf_plan **plan, const vdf_image_desc *descs, int count, int dist_mode, int minimax_q);
size_t vdf_plan_workspace_bytes(const vdf_plan *plan);
int vdf_plan_upload(vdf_plan *plan, void *workspace, size_t workspace_bytes, void *stream);
int vdf_filter_batch(vdf_plan *plan, void *workspace, size_t workspace_bytes, void *stream);
int vdf_plan_graph_launch(vdf_plan *plan, void *workspace, size_t workspace_bytes, void *stream);
int vdf_plan_set_persistent(vdf_plan *plan, int persistent);
void vdf_plan_destroy(vdf_plan *plan);

/*
 * Diagnostic: the FP32 path's per-member log scores and certified error
 * bounds, without selection.  fe_out: device, M*N*n*2 floats: f then E per
 * member.  BVDF: f is the aggregate.  DDF: f = (sum A)^(4p) (sum L2)^(4-4p)
 * (= Omega^4) when 4p is an integer, else f = p log2 sum A + (1-p) log2
 * sum L2.  The true value of f lies in [f - E, f + E].  Windows 3 and 5
 * (VDF_E_UNSUPPORTED for 7).
 */
int vdf_debug_fp32_scores(const uint8_t *img, int M, int N, int win, int filter, double p, int dist_mode,
                          int minimax_q, float *fe_out, void *stream);

/*
 * Diagnostic: the FP32 pair terms of n pixel pairs, exactly as the FP32 tile
 * kernel computes them before summing (the paper defines the terms in
 * Eq. (2) (arccos of the normalised inner product), Table 1 (Method 1,
 * degree minimax_q) and Eq. (7) (Method 2); it has no such call).  The FP32
 * path's certified bounds rest on these terms' error bounds: relative 16u
 * (arccos), 11u (Method 2), absolute 24u (Method 1), relative 5u (|x - y|),
 * u = 2^-24.
 *   pairs      device, n x 6 ints: R, G, B of x then of y, each in [0, 255]
 *              (other values give unspecified terms, never a fault)
 *   angle_out  device, n floats, or NULL: the angular term of dist_mode
 *   l2_out     device, n floats, or NULL: |x - y|
 * Errors: VDF_E_INVALID for a null pairs pointer, n < 0, or a bad dist_mode
 * or minimax_q; n = 0 launches nothing.  Asynchronous on stream.
 */
int vdf_debug_fp32_terms(const int *pairs, int n, int dist_mode, int minimax_q, float *angle_out, float *l2_out,
                         void *stream);

/*
 * Diagnostic: the FP32 exact-mode terms of n pairs of float pixels as the
 * float32-input FP32 tile kernel computes them (exponent-normalised pixels,
 * Kahan cross products; Eq. (2) and |x - y|).  pairs: device, n x 6 floats
 * (x then y, raw values); angle_out, l2_out: device, n floats each, or NULL;
 * NaN for a pair with an unsafe pixel (see vdf_filter_f32).  Bounds the path
 * relies on: angle relative 24u, L2 relative 8u, plus absolute 2^-58 and
 * 2^-62 where a product underflows.  The paper has no such call.
 * Errors: VDF_E_INVALID for null pairs or n < 0.
 */
int vdf_debug_fp32_terms_f32(const float *pairs, int n, float *angle_out, float *l2_out, void *stream);

/*
 * Diagnostic: the largest relative error, in units of u = 2^-24, of the
 * approximate square root the FP32 L2 terms use, over every positive normal
 * float (about 2.1e9 evaluations).  max_rel_err_u: device, one float,
 * written asynchronously on stream.  The paper has no such call.
 * Errors: VDF_E_INVALID for a null pointer.
 */
int vdf_debug_sqrt_error(float *max_rel_err_u, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* VDF_H */
