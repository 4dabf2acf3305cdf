/*
 * gs.h - C ABI of the B300 (sm_103a) differentiable Gaussian-splatting path
 * of GS-LIVO (arXiv 2501.08672).
 *
 * The library renders a sliding window of 3D Gaussians into one or more
 * keyframe views and back-propagates a photometric loss to the Gaussian
 * attributes (window map optimisation, Sec. II-B.2) and to the camera pose
 * (photometric pose update, Sec. II-D and Appendix A).  One iteration is
 *
 *   gs_project -> gs_bin -> gs_render_fwd -> gs_l1_loss -> gs_render_bwd
 *   (or gs_render_fwd_l1 for the middle two in one pass)
 *   -> gs_adam_step
 *
 * and the odometry form replaces the last two by gs_pose_grad.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers named *_dev, and every array pointer inside gs_gaussians,
 *   gs_grads and gs_workspace, are DEVICE pointers on the context's device.
 *   gs_view arrays and gs_config are HOST memory, read during the call only.
 * - Every call is asynchronous and stream-ordered on the given stream
 *   (a cudaStream_t; NULL is the legacy default stream).  No call allocates
 *   device memory, synchronises or copies to the host, except
 *   gs_context_create / gs_context_destroy (allocate / free a small status
 *   block), gs_sync_status and gs_bin with a non-NULL pairs_needed (both
 *   synchronise the stream).  Hence a whole iteration can be captured in a
 *   CUDA graph once gs_workspace_query has sized the workspace.
 * - The caller owns every buffer it passes.  A context is not thread-safe;
 *   use one context per host thread.
 * - Return value: GS_OK (0) or a negative gs_status.  Argument errors are
 *   detected on the host before anything is launched.  Errors found on the
 *   device (pair-capacity overflow) are latched in the context and reported
 *   by gs_sync_status.  No C++ exception crosses this interface and nothing
 *   aborts the process.  gs_last_error returns a message for the last error.
 *
 * Geometry (Sec. II-B.1, Eqs. 3dgs, q, spat)
 * ------------------------------------------
 * - Camera: p_C = R_CW p_W + t_CW; x right, y down, z forward; pinhole
 *   q = (fx x/z + cx, fy y/z + cy); pixel (u, v) is sampled at its centre
 *   (u + 0.5, v + 0.5).
 * - Gaussian: mean p_W; Sigma3 = R(q) S S^T R(q)^T with S = diag(exp(s)) and
 *   R(q) the rotation of the normalised quaternion (w, x, y, z);
 *   Sigma2 = J R_CW Sigma3 R_CW^T J^T + blur I with J the Jacobian of the
 *   pinhole map; opacity sigmoid(o); colour from real spherical harmonics of
 *   degree D <= 3 along the unit direction d from the camera centre to the
 *   mean: c = max(0, sum_k Y_k(d) k_k + 0.5), Y_k (k = l^2 + l + m,
 *   m = -l..l) the real harmonics with the Condon-Shortley phase; degree 1
 *   reads c = max(0, C0 k0 + C1 (-d_y k1 + d_z k2 - d_x k3) + 0.5).
 * - Compositing (Eq. raster): per pixel, front to back over the Gaussians
 *   ordered by (depth, index): alpha = min(alpha_max, sigma G(x)); skip if
 *   alpha < alpha_min; stop before the Gaussian that would take the
 *   transmittance below T_min; C += c alpha T; T *= 1 - alpha.  Output
 *   C + T bg.  The set of Gaussians tested at a pixel is every Gaussian
 *   whose alpha can reach alpha_min there, so the image does not depend on
 *   the tile size.
 */
#ifndef GS_B300_GS_H
#define GS_B300_GS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Symbols of this interface are exported; everything else in the library is
 * hidden. */
#if defined(__GNUC__)
#define GS_API __attribute__((visibility("default")))
#else
#define GS_API
#endif

/* Opaque CUDA stream handle (a cudaStream_t). */
typedef struct CUstream_st* gs_stream;

typedef enum gs_status {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = -1, /* bad pointer, size, dtype, view or config */
    GS_ERR_CUDA = -2,        /* a CUDA runtime call or launch failed */
    GS_ERR_OOM = -3,         /* context status block could not be allocated */
    GS_ERR_CAPACITY = -4,    /* more (Gaussian, tile) pairs than the workspace holds */
    GS_ERR_TIMEOUT = -5,     /* a bounded device wait expired (latched, see gs_sync_status) */
    GS_ERR_NONFINITE = -6,   /* a camera or intrinsic value is not finite */
    GS_ERR_UNSUPPORTED = -7, /* option not built into this library */
    GS_ERR_BOUNDS = -8       /* checked build only: an index read from device memory failed its bounds
                                check and the access was skipped (latched, see gs_sync_status) */
} gs_status;

typedef enum gs_dtype { GS_F32 = 0, GS_F16 = 1, GS_BF16 = 2 } gs_dtype;

#define GS_MAX_VIEWS 64

/* Rasteriser constants.  gs_config_default fills the defaults in brackets
 * (the constants of the 3D-GS tile rasteriser the paper builds on,
 * Sec. II-C).  alpha_min = 0, alpha_max = 1, T_min = 0 gives Eq. raster
 * literally ("exact mode"). */
typedef struct gs_config {
    int32_t tile_size; /* 8, 16 or 32 [16] */
    float alpha_min;   /* [1/255] */
    float alpha_max;   /* [0.99] */
    float T_min;       /* [1e-4] */
    float blur;        /* low-pass term added to the diagonal of Sigma2, px^2 [0.3] */
    float z_near;      /* Gaussians with camera depth <= z_near are culled, m [0.2] */
    float bg[3];       /* background colour [0, 0, 0] */
    /* Launch shape of the compositing kernels (0 = default).  pixels_per_thread:
     * 1, 2 for tile 8; 1, 2, 4, 8 for tile 16; 4, 8 for tile 32 [2, 2, 4];
     * batch: records staged per shared-memory batch, 128 or 256, at least the
     * threads per tile (tile^2 / pixels_per_thread) [128 up to 128 threads per
     * tile, else 256].  The result does not depend on them; the defaults are
     * the fastest measured at the headline workload, and render.autotune
     * times the compiled shapes for a given workload. */
    int32_t pixels_per_thread;
    int32_t batch;
    /* 1: gs_render_bwd sums every gradient in a fixed order, so the same
     * inputs give the same gradients bit for bit on every run [0].  Each
     * tile's warps add their per-record totals in shared memory in warp
     * order, one 9-float partial per (tile, record) pair is written at the
     * pair's place in the tile lists, and each record's partials are added in
     * the order of its tiles; the default adds the totals with float atomics,
     * whose order varies.  Costs 56 bytes of workspace per pair of capacity
     * (gs_workspace_query includes them) and some speed. */
    int32_t deterministic;
    /* Tile size of the binning (a2) [0 = tile_size].  2 or 4 times
     * tile_size, at most 32: gs_project and gs_bin list and sort the records
     * per bin of F x F tiles (F = bin_tile_size / tile_size), which has
     * fewer (bin, record) pairs to sort than (tile, record) pairs, and gs_bin
     * then splits each bin's front-to-back list, keeping its order, into the
     * lists of the bin's F^2 tiles, a record going to each tile its
     * alpha >= alpha_min footprint reaches (the binning's own row-span test
     * at tile_size, so each tile gets the list that binning at tile_size
     * gives).  The compositing kernels read those per-tile lists.  Used in
     * truncated mode (alpha_min > 0) without deterministic only; otherwise the
     * binning runs at tile_size, and likewise when the batch has 2^(32 - F^2)
     * - 1 bins or more (the pair keys hold the bin id below the F^2-bit tile
     * mask).  Costs 4 F^2 bytes of workspace per pair of capacity (max_pairs
     * then counts (bin, record) pairs, and F^2 max_pairs must stay below
     * 2^32).  8 x 8 tiles from 32 x 32 bins is the fastest measured at the
     * headline workload. */
    int32_t bin_tile_size;
} gs_config;

GS_API void gs_config_default(gs_config* cfg);

typedef struct gs_ctx gs_ctx;

/* Creates a context on CUDA device `device` (made current for the call).
 * cfg may be NULL for the defaults.  Allocates a small device status block.
 * Errors: GS_ERR_INVALID_ARG (out NULL, bad config), GS_ERR_CUDA, GS_ERR_OOM. */
GS_API int gs_context_create(gs_ctx** out, int device, const gs_config* cfg);
/* Frees the context and its status block.  NULL is accepted. */
GS_API int gs_context_destroy(gs_ctx* ctx);
/* Message of the last error on this context ("" if none); valid until the
 * next call on the context. */
GS_API const char* gs_last_error(const gs_ctx* ctx);
/* Copies the context's configuration into *cfg. */
GS_API int gs_get_config(const gs_ctx* ctx, gs_config* cfg);

/* One keyframe view (host memory).  The view renders the contiguous Gaussian
 * range [g_begin, g_end) of the window, mirroring the paper's contiguous GPU
 * Gaussian buffer (Sec. II-C); 0 <= g_begin < g_end <= n is required.  Views are
 * packed one after another in every per-pixel and per-record buffer in the
 * order given: view v's pixels start at pixel offset sum_{u<v} W_u H_u, its
 * projected records at sum_{u<v} (g_end_u - g_begin_u). */
typedef struct gs_view {
    float R_cw[9]; /* camera-from-world rotation, row-major */
    float t_cw[3]; /* camera-from-world translation */
    float fx, fy, cx, cy;
    int32_t width, height;
    int64_t g_begin, g_end;
} gs_view;

/* The Gaussian window (device memory, structure of arrays, row-major).
 * means is always FP32; the other fields may be stored in FP16 or BF16
 * (all arithmetic is FP32). */
typedef struct gs_gaussians {
    const float* means;     /* [N,3] world metres */
    const void* log_scales; /* [N,3] log of the standard deviations */
    const void* quats;      /* [N,4] (w, x, y, z), need not be normalised */
    const void* opacity;    /* [N] logit of the opacity */
    const void* sh;         /* [N,K,3], K = (sh_degree+1)^2, coefficient-major */
    int32_t scale_dtype, rot_dtype, opacity_dtype, sh_dtype; /* gs_dtype */
    int64_t n;
    int32_t sh_degree; /* 0 to 3 */
} gs_gaussians;

/* Gradients (device memory, FP32, same shapes as gs_gaussians).  Every entry
 * is overwritten, including Gaussians that no view sees (zero). */
typedef struct gs_grads {
    float* means;
    float* log_scales;
    float* quats;
    float* opacity;
    float* sh;
} gs_grads;

/* Caller-allocated device workspace holding the projected records, the
 * sorted (tile, depth) pairs, the per-tile ranges and the per-record 2D
 * gradients of one batch of views.  `bytes` must be at least what
 * gs_workspace_query returned for the same views and max_pairs; the base
 * pointer must be 256-byte aligned (cudaMalloc and torch allocations are). */
typedef struct gs_workspace {
    void* ptr;
    size_t bytes;
    int64_t max_pairs; /* capacity for (Gaussian, tile) pairs */
} gs_workspace;

/* Byte offsets of the workspace arrays, for inspection and tests. */
typedef struct gs_ws_layout {
    size_t records;       /* float[M][12]: qx, qy, v1x, v1y, v2x, v2y, log2(opacity), r, g, b, depth, 0 */
    size_t rects;         /* int32[M][8]: x0|y0<<16, x1|y1<<16, first tile id of the view, tiles_x,
                           * tiles touched, mask of the listed tiles (row-major over the rectangle when it
                           * has at most 32 tiles, else 0), 0, 0 */
    size_t tiles_touched; /* uint32[M] */
    size_t depth_keys;    /* uint32[M] low words of the 64-bit depth keys, record order (two buffers) */
    size_t depth_hi;      /* uint32[M] high words of the 64-bit depth keys (overwritten by gs_bin's sort) */
    size_t depth_vals;    /* uint32[M] record indices (two buffers) */
    size_t pair_offsets;  /* uint64[M] */
    size_t pair_keys;     /* uint32[max_pairs] x 2 (binning at a larger bin size: the bin id in the low
                             32 - F^2 bits, the mask of its tiles the footprint reaches above) */
    size_t pair_vals;     /* uint32[max_pairs] x 2 */
    size_t sorted_vals;   /* the buffer holding the sorted record index per pair */
    size_t tile_ranges;   /* uint32[T][2] [start, end) into sorted_vals */
    size_t grad2d;        /* float[M][9] per-record 2D gradients */
    size_t counters;      /* uint64[8]: [0] pairs needed; [1..3] the projection's depth-key range and its generation */
    size_t total;         /* bytes */
    int64_t n_records;    /* M */
    int32_t n_tiles;      /* T (tiles of the compositing) */
    int64_t n_pixels;
    /* Binning at a larger bin size (gs_config.bin_tile_size): rects,
     * tiles_touched and the pair arrays count bins; bin_vals holds the sorted
     * record index per (bin, record) pair, bin_ranges (uint32[n_bins][2])
     * each bin's [start, end) into it, and sorted_vals / tile_ranges the
     * per-tile lists split from them.  Otherwise bin_vals = sorted_vals,
     * bin_ranges = tile_ranges and n_bins = n_tiles. */
    size_t bin_keys;      /* the sorted pair keys (bin id, tile mask above it) */
    size_t bin_vals;
    size_t bin_ranges;
    int32_t n_bins;
    int32_t bin_size;     /* pixels per bin side (tile_size when not refined) */
} gs_ws_layout;

/* Workspace size for `n_views` views and a pair capacity max_pairs.
 * Errors: GS_ERR_INVALID_ARG. */
GS_API int gs_workspace_query(const gs_ctx* ctx, const gs_view* views, int n_views, int64_t max_pairs,
                       size_t* bytes);
GS_API int gs_workspace_layout(const gs_ctx* ctx, const gs_view* views, int n_views, int64_t max_pairs,
                        gs_ws_layout* out);

/* a1: EWA projection of every (view, Gaussian) pair (Sec. II-B.1, Eqs. 3dgs,
 * q, spat; colour from SH; opacity sigmoid).  Writes the projected records,
 * tile rectangles and tiles-touched counts into the workspace.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_NONFINITE, GS_ERR_CUDA. */
GS_API int gs_project(gs_ctx* ctx, const gs_gaussians* g, const gs_view* views, int n_views,
               const gs_workspace* ws, gs_stream stream);

/* a2: tile binning.  Orders the records front to back (radix sort of the
 * FP32 depth bits, stable in record index), expands each record into one
 * pair per tile its footprint touches, and stably radix-sorts the pairs by
 * global tile id, so each tile's list is ordered by (depth, index): the
 * order a radix sort of 64-bit (tile << 32 | depth) keys gives.  Then
 * extracts each tile's [start, end) range.  The tile sort is implied by the
 * 3D-GS rasteriser the paper relies on (Sec. II-C).  With
 * gs_config.bin_tile_size above the tile size the records are binned and
 * sorted per bin of F x F tiles, and each bin's list is then split, in
 * order, into its tiles' lists (the pair count and capacity then count
 * (bin, record) pairs).
 * pairs_needed: NULL (fully asynchronous) or a host pointer that receives
 * the number of pairs after a stream synchronisation.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA; with pairs_needed non-NULL also
 * GS_ERR_CAPACITY when the pairs exceed ws->max_pairs (the render is then
 * incomplete; call again with a larger workspace). */
GS_API int gs_bin(gs_ctx* ctx, const gs_view* views, int n_views, const gs_workspace* ws,
           uint64_t* pairs_needed, gs_stream stream);

/* a3: front-to-back alpha compositing (Sec. II-B.2, Eq. raster), one CTA per
 * tile over the tile's sorted list, staged in shared memory, stopping early
 * once every pixel's transmittance is below T_min.
 * Outputs (device, packed over views): rgb [sum 3 H W] (view v planar
 * [3,H,W]), T_final [sum H W], n_contrib [sum H W] (1 + position in the
 * tile's list of the last contributing Gaussian, 0 if none; consumed by
 * gs_render_bwd), n_used [sum H W] (number of contributing Gaussians; may be
 * NULL).  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
GS_API int gs_render_fwd(gs_ctx* ctx, const gs_view* views, int n_views, const gs_workspace* ws,
                  float* rgb, float* T_final, uint32_t* n_contrib, uint32_t* n_used,
                  gs_stream stream);

/* a3 + a4 in one pass: the compositing of gs_render_fwd with the L1 loss of
 * gs_l1_loss folded into it (Eq. gaussian_optimization): each pixel's
 * gradient needs only its own colour and target, so the compositing kernel
 * writes dL_drgb as it finishes a pixel, and one partial sum per tile that a
 * second launch adds up into loss_dev[0].  Same values as gs_render_fwd
 * followed by gs_l1_loss: rgb, T_final, n_contrib, n_used and dL_drgb bit for
 * bit; the loss up to the order of the FP32 sum.
 * target: device FP32, packed like rgb.  rgb: may be NULL (the image is then
 * not written; the loss and gradient are).  n_used, loss_dev: may be NULL.
 * The per-tile partials live in the workspace.
 * Errors: GS_ERR_INVALID_ARG (target, T_final, n_contrib or dL_drgb NULL),
 * GS_ERR_CUDA. */
GS_API int gs_render_fwd_l1(gs_ctx* ctx, const gs_view* views, int n_views, const gs_workspace* ws,
                            const float* target, float* rgb, float* T_final, uint32_t* n_contrib,
                            uint32_t* n_used, float* dL_drgb, float* loss_dev, gs_stream stream);

/* Device floats of scratch gs_dssim_loss needs for these views: 9 per pixel
 * (three SSIM derivative maps per channel) plus one per 32 x 16 tile of each
 * channel; 0 if the views are invalid. */
GS_API size_t gs_dssim_scratch_floats(const gs_view* views, int n_views);

/* Photometric loss with a structural term (the paper's Eq.
 * gaussian_optimization uses the L1 norm; this is the D-SSIM variant common
 * in 3D-GS training):
 *   L = (1/V) sum_v [(1 - lambda) mean_{3 H_v W_v} |x - y| + lambda (1 - mean SSIM(x, y))]
 * with x = rgb, y = target (both packed over views like gs_render_fwd's
 * output), SSIM per channel with an 11 x 11 Gaussian window (sigma 1.5), zero
 * padding, C1 = 0.01^2, C2 = 0.03^2:
 *   SSIM = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_x^2 + s_y^2 + C2)).
 * Writes L to loss_dev[0] (may be NULL) and dL/drgb to dL_drgb.  lambda in
 * [0, 1]; lambda = 0 is gs_l1_loss.  scratch: device, caller-owned,
 * gs_dssim_scratch_floats(views, n_views) floats, 16-byte aligned.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
GS_API int gs_dssim_loss(gs_ctx* ctx, const gs_view* views, int n_views, const float* rgb, const float* target,
                         float lambda, float* scratch, float* dL_drgb, float* loss_dev, gs_stream stream);

/* a4: photometric loss (Eq. gaussian_optimization, L1 norm):
 * L = (1/V) sum_v mean_{3 H_v W_v} |rgb - target| written to loss_dev[0], and
 * dL/drgb = sign(rgb - target) / (3 H_v W_v V) written to dL_drgb (sign(0) = 0).
 * loss_dev may be NULL.  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
GS_API int gs_l1_loss(gs_ctx* ctx, const gs_view* views, int n_views, const gs_workspace* ws,
               const float* rgb, const float* target, float* dL_drgb, float* loss_dev,
               gs_stream stream);

/* a5 + a6 (+ a7): backward of the compositing (reverse order from n_contrib,
 * alpha recomputed, transmittance recovered by division) into per-record 2D
 * gradients, then backward of the projection to every Gaussian parameter
 * (summed over views) and, if dL_dpose_dev is non-NULL, to each view's pose.
 * dL_dpose_dev: [n_views][6] = dL/d(dphi_x, dphi_y, dphi_z, dt_x, dt_y, dt_z)
 * for the left perturbation T_CW <- Exp(dphi, dt) T_CW (Appendix A,
 * perturbation model).  grads may be NULL only when dL_dpose_dev is not.
 * Clamped alpha and colour, culling and the footprint are locally constant.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
GS_API int gs_render_bwd(gs_ctx* ctx, const gs_gaussians* g, const gs_view* views, int n_views,
                  const gs_workspace* ws, const float* T_final, const uint32_t* n_contrib,
                  const float* dL_drgb, const gs_grads* grads, float* dL_dpose_dev,
                  gs_stream stream);

/* gs_render_bwd, with the parameter gradients added to what grads already
 * holds instead of overwriting it (every entry of every group, zero for
 * Gaussians no view of this call sees).  The window optimisation of
 * Sec. II-B.2 takes one Adam step on the gradient of a loss summed over the
 * keyframes (Eq. gaussian_optimization over the window's images); this form
 * lets that gradient be formed over several calls (more views than
 * GS_MAX_VIEWS, or one view per launch sequence) before the one Adam step.  The gradients of the first call's Gaussians must be
 * cleared (or written by gs_render_bwd) first.  dL_dpose_dev, when non-NULL,
 * is written per view as in gs_render_bwd.  grads is required.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
GS_API int gs_render_bwd_accumulate(gs_ctx* ctx, const gs_gaussians* g, const gs_view* views, int n_views,
                                    const gs_workspace* ws, const float* T_final, const uint32_t* n_contrib,
                                    const float* dL_drgb, const gs_grads* grads, float* dL_dpose_dev,
                                    gs_stream stream);

/* a7: photometric pose gradient only (Sec. II-D, Eq. minimization; the
 * derivative chain of Eqs. grad_meani_rcw to grad_covi_tcw restricted to the
 * camera pose): gs_render_bwd with grads = NULL.  dL_dpose_dev is required. */
GS_API int gs_pose_grad(gs_ctx* ctx, const gs_gaussians* g, const gs_view* views, int n_views,
                 const gs_workspace* ws, const float* T_final, const uint32_t* n_contrib,
                 const float* dL_drgb, float* dL_dpose_dev, gs_stream stream);

/* Optional low-precision render copy written by gs_adam_step: elements
 * [begin, end) of the FP32 parameter vector are also stored, converted to
 * `dtype`, at dst[i - begin]. */
typedef struct gs_lowp_segment {
    int64_t begin, end;
    int32_t dtype; /* GS_F16 or GS_BF16 */
    void* dst;
} gs_lowp_segment;

/* a8: one Adam step (Sec. II-B.2, "Adam optimizer"; Kingma & Ba with bias
 * correction, the update rule of torch.optim.Adam) over n FP32 parameters in
 * place: m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
 * p -= lr / (1 - b1^step) * m / (sqrt(v) / sqrt(1 - b2^step) + eps).
 * step >= 1.  segs: up to 8 low-precision copies (may be NULL).
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
GS_API int gs_adam_step(gs_ctx* ctx, float* param, const float* grad, float* m, float* v, int64_t n,
                 float lr, float b1, float b2, float eps, int64_t step,
                 const gs_lowp_segment* segs, int n_segs, gs_stream stream);

/* a8, graph-friendly form: as gs_adam_step, but the step count lives in
 * device memory.  step_dev (device, int64) holds the number of steps already
 * taken; the call increments it on the stream and uses the new value for the
 * bias correction, so one captured launch sequence advances it on every
 * replay.  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
GS_API int gs_adam_step_dev(gs_ctx* ctx, float* param, const float* grad, float* m, float* v, int64_t n,
                            float lr, float b1, float b2, float eps, int64_t* step_dev,
                            const gs_lowp_segment* segs, int n_segs, gs_stream stream);

/* An element range [begin, end) of a flat parameter vector. */
typedef struct gs_range {
    int64_t begin, end;
} gs_range;

/* a8 over the active rows only: the Adam step of gs_adam_step applied to the
 * elements of up to 8 disjoint ranges of the n-element buffers (begin a
 * multiple of 4, end <= n; the buffers 16-byte aligned), e.g. rows [0, n_g)
 * of each parameter group of a window with spare capacity, so that rows
 * outside the ranges (Gaussians being appended on another stream) are never
 * read or written.  With step_dev non-NULL the step count lives on the
 * device as in gs_adam_step_dev (step is ignored); else step >= 1 is used.
 * Low-precision segments as in gs_adam_step (written for elements inside
 * the ranges).  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
GS_API int gs_adam_step_ranges(gs_ctx* ctx, float* param, const float* grad, float* m, float* v, int64_t n,
                               const gs_range* ranges, int n_ranges, float lr, float b1, float b2, float eps,
                               int64_t step, int64_t* step_dev, const gs_lowp_segment* segs, int n_segs,
                               gs_stream stream);

/* L1 loss that allocates nothing and needs no context or workspace.  The
 * paper has no counterpart: this entry point exists for callers that cannot
 * allocate device memory, such as a real-time loop that allocates nothing
 * after start-up so that no allocation can stall or fail mid-run, or a host
 * framework that owns every device allocation itself.
 * It computes what gs_l1_loss computes (same arguments, without ctx and ws),
 * on the current CUDA device.  Its per-block partial sums live in a fixed
 * 1 MiB array inside the library's device memory (loaded on every GPU that
 * uses the library and kept until the process exits), so
 *   n_views * ceil(3 * max_v(W_v * H_v) / 1024) <= 262144
 * is required, e.g. 64 views of 1280 x 1024; larger batches return
 * GS_ERR_CAPACITY with a message in msg.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture on that device.  The address belongs to the CUDA
 * context it was looked up in: the first call in a new context on the device
 * (after cudaDeviceReset, for instance) looks it up again, and that call too
 * must come before any stream capture (a captured one returns
 * GS_ERR_INVALID_ARG).  `stream` must belong to the current device
 * (GS_ERR_INVALID_ARG otherwise).  All calls on a device share the array:
 * calls whose work overlaps on the GPU (for instance on two streams) race and
 * must be ordered by the caller.  Each call rewrites every slot it reads, so
 * nothing needs clearing between calls.
 * msg: NULL or a host buffer of msg_len bytes that receives an error text.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CAPACITY, GS_ERR_CUDA. */
GS_API int gs_l1_loss_noalloc(const gs_view* views, int n_views, const float* rgb, const float* target,
                              float* dL_drgb, float* loss_dev, gs_stream stream, char* msg,
                              size_t msg_len);

/* Synchronises `stream`, returns and clears the latched device status
 * (GS_OK, GS_ERR_CAPACITY, or GS_ERR_TIMEOUT when a bounded wait of the
 * binning's single-pass scan expired and its result is unusable); pairs_needed (nullable, host) receives the
 * pair count of the last gs_bin on this context. */
GS_API int gs_sync_status(gs_ctx* ctx, gs_stream stream, uint64_t* pairs_needed);

/* Failure-detection self-test.  Runs the binning's single-pass scan on two
 * chunks of `scratch` (device, gs_selftest_wait_scratch_bytes() bytes,
 * 256-byte aligned, caller-owned) with its ticket started past the first
 * chunk, so the one block waits for a flag that nothing sets; its bounded
 * wait expires (about a second at most) and the device latches
 * GS_ERR_TIMEOUT, which the next gs_sync_status returns and clears.  Nothing
 * faults and the context stays usable.  Errors: GS_ERR_INVALID_ARG,
 * GS_ERR_CUDA. */
GS_API size_t gs_selftest_wait_scratch_bytes(void);
GS_API int gs_selftest_bounded_wait(gs_ctx* ctx, void* scratch, gs_stream stream);

/* Kernel families, for profiling (bit i of a mask selects family i). */
typedef enum gs_kernel_family {
    GS_KF_PROJECT = 0,     /* a1 projection */
    GS_KF_DEPTH_SORT = 1,  /* a2 radix sort of record depths */
    GS_KF_TILE_SCAN = 2,   /* a2 scan of tiles touched */
    GS_KF_EMIT = 3,        /* a2 pair emission */
    GS_KF_TILE_SORT = 4,   /* a2 radix sort of pairs by tile */
    GS_KF_RANGES = 5,      /* a2 tile ranges */
    GS_KF_RASTER_FWD = 6,  /* a3 compositing */
    GS_KF_L1 = 7,          /* a4 loss */
    GS_KF_RASTER_BWD = 8,  /* a5 compositing backward */
    GS_KF_PROJECT_BWD = 9, /* a6/a7 projection backward and pose reduction */
    GS_KF_ADAM = 10,       /* a8 Adam */
    GS_KF_POSE_NORMAL = 11, /* pose tangents, forward-mode compositing, normal equations */
    GS_KF_WINDOW = 12,      /* sliding-window maintenance and SH0 initialisation */
    GS_KF_SSIM = 13,        /* photometric loss with the D-SSIM term */
    GS_KF_REFINE = 14,      /* a2 split of the bin lists into tile lists */
    GS_KF_COUNT = 15
} gs_kernel_family;

typedef struct gs_profile_entry {
    int32_t family;   /* gs_kernel_family */
    int32_t launches; /* timed launches since the last collect */
    double total_ms;  /* summed CUDA-event time of those launches */
} gs_profile_entry;

/* Tracing: when bit f of family_mask is set, every launch of family f is
 * bracketed by CUDA events on its stream (events are created on first use,
 * outside any stream capture; disable profiling before capturing a graph).
 * 0 disables.  Errors: GS_ERR_INVALID_ARG. */
GS_API int gs_profile_enable(gs_ctx* ctx, uint32_t family_mask);
/* Synchronises `stream`, writes one entry per family with timed launches
 * (at most max_entries) and clears the record.  *n_out receives the count. */
GS_API int gs_profile_collect(gs_ctx* ctx, gs_stream stream, gs_profile_entry* out, int max_entries,
                              int* n_out);
/* Number of kernel launches (and memset nodes) this context has issued. */
GS_API int64_t gs_launch_count(const gs_ctx* ctx);
/* 1 in the checked build of the library (libgs_b300_checked.so, compiled
 * with GS_CHECKED: the compositing kernels bounds-check every tile range and
 * pair record they read and latch GS_ERR_BOUNDS instead of reading out of
 * bounds), 0 in the normal build.  Same API and results otherwise. */
GS_API int32_t gs_checked_build(void);

/* ---- pose normal equations of the photometric residual (Sec. II-D) ----
 *
 * The visual update of the paper's iterated error-state Kalman filter
 * (Sec. II-D, Eq. minimization; Appendix A) linearises the rendered image in
 * the camera pose.  For each view this computes, over every pixel x and
 * channel ch, with H_ch(x) = dI_ch(x)/dxi the 6-vector derivative of the
 * rendered colour with respect to the left perturbation xi = [dphi; dt],
 * T_CW <- Exp(xi) T_CW, and r_ch(x) = target_ch(x) - I_ch(x):
 *   normal[v][0..20]  = upper triangle of A = sum H H^T, row-major
 *                       ((0,0), (0,1), ..., (0,5), (1,1), ..., (5,5)),
 *   normal[v][21..26] = b = sum H r,
 *   normal[v][27]     = sum r^2,
 * so that the Gauss-Newton step of the pose is xi = A^-1 b.  H is obtained
 * by forward-mode differentiation of Eq. raster through Eqs. q and spat and
 * the view direction of the SH colour; culling and the set of contributing
 * fragments are locally constant, clamped alphas and colours contribute zero
 * derivative.  The per-tile sums are FP32, the per-view sums FP64 (in a
 * fixed order: 64 runs of tiles per view, then the runs).
 *
 * Requires gs_project and gs_bin on the same views and workspace (as
 * gs_render_fwd) and a tile size of 8 or 16 (GS_ERR_UNSUPPORTED otherwise).
 * target: device FP32, packed like rgb of gs_render_fwd.  scratch: device
 * FP32 of gs_pose_normal_scratch() floats, 16-byte aligned, caller-owned,
 * overwritten.  normal: device FP64 [n_views][28].  H_pix: NULL, or device
 * FP32 [total pixels][3][6] (packed over views like T_final) receiving H.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_UNSUPPORTED, GS_ERR_CUDA. */
GS_API int gs_pose_normal_scratch(gs_ctx* ctx, const gs_view* views, int n_views, size_t* floats);
GS_API int gs_pose_normal(gs_ctx* ctx, const gs_gaussians* g, const gs_view* views, int n_views,
                          const gs_workspace* ws, const float* target, float* scratch, double* normal,
                          float* H_pix, gs_stream stream);

/* ---- sliding-window maintenance on the device (Sec. II-C) ----
 *
 * The window's per-Gaussian data are columns: column c holds
 * bytes_per_gaussian bytes for every Gaussian (a multiple of 4, at most
 * GS_WINDOW_MAX_COLUMN_BYTES), Gaussian i at ptr + i * bytes_per_gaussian
 * (device, 4-byte aligned).  The FP32 parameter groups, the Adam moments and
 * the FP16/BF16 render copies are all columns. */
#define GS_WINDOW_MAX_COLUMN_BYTES 16384
typedef struct gs_window_column {
    void* ptr;
    int32_t bytes_per_gaussian;
} gs_window_column;

/* Device scratch bytes gs_window_compact needs for a window of n rows. */
GS_API size_t gs_window_scratch_bytes(int64_t n);

/* Step 2 of the window maintenance (deletion and compaction, Sec. II-C):
 * removes the rows whose keep[i] is 0 by swapping survivors from the rear
 * into the holes.  With n_keep survivors, the k-th hole (a removed row below
 * n_keep, ascending) receives the k-th surviving row at or above n_keep
 * counted from the rear (descending); survivors below n_keep do not move, so
 * afterwards the window is rows [0, n_keep).  keep: device uint8[n].
 * n_keep_dev: device int64, receives n_keep.  moved_from: NULL or device
 * int32[n]; for every row r < n_keep it receives the row whose data r now
 * holds (r itself if unmoved); rows >= n_keep are left as they were.
 * scratch: device, gs_window_scratch_bytes(n) bytes, caller-owned.  At most 32
 * columns.  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
GS_API int gs_window_compact(gs_ctx* ctx, const gs_window_column* cols, int n_cols, int64_t n, const uint8_t* keep,
                             int64_t* n_keep_dev, int32_t* moved_from, void* scratch, gs_stream stream);

/* Steps 1 and 2 in one stream-ordered call, without host synchronisation:
 * the rows whose keep[i] is 0 are (1) gathered in ascending row order into
 * rows 0, 1, ... of leave_dst (the copy of leaving Gaussians to the global
 * map; a NULL column pointer skips that column, leave_dst NULL skips the
 * gather) and (2) removed by the compaction of gs_window_compact.  The
 * number of leaving rows is n - n_keep (n_keep_dev receives n_keep); every
 * leave_dst column must have room for n rows.  leaving_rows: NULL or device
 * int32[n]; its first n - n_keep entries receive the leaving rows ascending.
 * moved_from and scratch as gs_window_compact.  leave_dst columns have the
 * bytes_per_gaussian of the matching window column.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
GS_API int gs_window_remove(gs_ctx* ctx, const gs_window_column* cols, const gs_window_column* leave_dst, int n_cols,
                            int64_t n, const uint8_t* keep, int64_t* n_keep_dev, int32_t* moved_from,
                            int32_t* leaving_rows, void* scratch, gs_stream stream);

/* Step 1 copy-back: gathers rows idx[0..m) (device int32, each in [0, n))
 * of every src column into rows 0..m of the matching dst column (same
 * bytes_per_gaussian), for the copy of leaving Gaussians to the global map.
 * At most 32 columns.  Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
GS_API int gs_window_gather(gs_ctx* ctx, const gs_window_column* src, const gs_window_column* dst, int n_cols,
                            int64_t n, const int32_t* idx, int64_t m, gs_stream stream);

/* Step 4 insertion: sets rows [begin, end) of every column to zero (the
 * gradients and Adam moments of Gaussians entering the window).  The columns
 * must hold at least `end` rows.  At most 32 columns.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_CUDA. */
GS_API int gs_window_clear(gs_ctx* ctx, const gs_window_column* cols, int n_cols, int64_t begin, int64_t end,
                           gs_stream stream);

/* SH initialisation of new Gaussians (Sec. II-B.2): for Gaussians
 * [begin, end) of g, the colour c is the bilinear interpolation of `image`
 * (device FP32 [3, H, W] of `view`) at the projected mean, pixel (u, v)
 * sampled at (u + 0.5, v + 0.5), and the FP32 SH coefficients sh_out
 * ([n][(D+1)^2][3], D = g->sh_degree) get k0 = (c - 0.5) / C0 and 0 for the
 * higher orders.  A Gaussian behind z_near or projecting outside the image
 * gets c = 0.5 (k0 = 0).  g->means must be FP32.
 * Errors: GS_ERR_INVALID_ARG, GS_ERR_NONFINITE, GS_ERR_CUDA. */
GS_API int gs_sh_init_bilinear(gs_ctx* ctx, const gs_gaussians* g, const gs_view* view, const float* image,
                               int64_t begin, int64_t end, float* sh_out, gs_stream stream);

/* Measures, on the context's device, the throughput of the FP32 FMA pipe
 * (FLOP/s, an FMA counting 2) and of the ex2 special-function unit (ex2/s)
 * with two short microbenchmarks (a few ms each, best of 3), the measured
 * ALU peaks that the compositing kernels' roofline is quoted against.  Not
 * part of the rendering path; synchronises `stream`.
 * Errors: GS_ERR_INVALID_ARG (NULL output), GS_ERR_CUDA. */
GS_API int gs_calibrate_alu(gs_ctx* ctx, gs_stream stream, double* ffma_tflops, double* ex2_gops);

/* Library version string. */
GS_API const char* gs_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GS_B300_GS_H */
