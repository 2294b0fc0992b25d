/*
 * gps.h - C ABI of the Gaussian-plus-SDF hot path (libgps.so, sm_103a).
 *
 * The library implements the per-frame Gaussian-overlay optimisation of
 * Gaussian-plus-SDF reconstruction (arXiv 2509.11574): colourised TSDF fusion
 * and SDF ray-casting (Sec. 3.1, Sec. 3.2.1) as supporting steps, then the
 * hybrid render of Eq. 1-4 (or the sorted "with sort" variant of Table 7), the
 * L1 loss (Eq. 6), its adjoint to every Gaussian parameter, and an Adam step
 * with the learning rates of App. C.
 *
 * Conventions shared by every call
 *   - All functions return int32_t status (GPS_OK = 0, negative on error) and
 *     never throw.  On error `gps_last_error()` (thread-local) describes it.
 *   - Device pointers are CUDA device addresses owned by the caller.  The
 *     library allocates no device memory: scratch comes from a caller-provided
 *     workspace sized by `gps_workspace_size`.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Every call only enqueues work on it and performs no host
 *     synchronisation, so calls can be captured into a CUDA graph.
 *     Errors discovered on the device (pair-buffer overflow, a bounded wait
 *     that ran out) are recorded in the workspace status word and read with
 *     `gps_query_status` after the stream has been synchronised.
 *   - Camera frame: x right, y down, +z forward.  A pose is camera->world:
 *     X_w = R X_c + t with R row-major, t the camera centre.  Pixel (i, j)
 *     (column i, row j) has its centre at image coordinate (i, j):
 *     u = fx x / z + cx.  Images are planar float32 [C][H][W]; depth is camera
 *     z in metres, 0 = invalid / no surface.
 *   - Gaussian parameters are float32 arrays: means [M][3], log_scales [M][3],
 *     quats [M][4] (w, x, y, z; normalised inside), opacity_logits [M]
 *     (sigma = sigmoid(logit)), rgb [M][3], and optionally spherical-harmonic
 *     coefficients sh_rest [M][K][3] of degree 1..D (K = (D+1)^2 - 1, D <= 3).
 *     The colour seen from a camera centre o is
 *       c_i = rgb_i + sum_{l=1..D} sum_{m=-l..l} Y_lm(d) f_lm,  d = (p_i - o)/|p_i - o|,
 *     Y_lm the real orthonormal harmonics (Condon-Shortley phase; per l the
 *     coefficients are stored for m = -l..l), so with D = 0 the colour is rgb.
 */
#ifndef GPS_H_
#define GPS_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define GPS_API __attribute__((visibility("default")))
#else
#define GPS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define GPS_OK 0
#define GPS_ERR_INVALID_ARG (-1)         /* bad pointer, size or setting       */
#define GPS_ERR_WORKSPACE_TOO_SMALL (-2) /* ws_bytes < gps_workspace_size()     */
#define GPS_ERR_CAPACITY (-3)            /* more (super-tile, Gaussian) entries
                                            than pair_capacity (with tile bins:
                                            (tile, Gaussian) entries than
                                            tiles per super-tile times
                                            pair_capacity); found on the
                                            device */
#define GPS_ERR_CUDA (-4)                /* a CUDA launch / copy failed         */
#define GPS_ERR_TIMEOUT (-5)             /* a bounded device wait gave up       */

/* blend modes of the second rendering pass */
#define GPS_BLEND_OIT 0   /* Eq. 1-4: order-independent, depth-culled, W_t = 1   */
#define GPS_BLEND_ALPHA 1 /* Table 7 "with sort": front-to-back alpha over C_t  */

/* storage type of the colour images: C_t (GpsView.sdf_rgb, raycast_sdf's
   out_rgb), the observed colour C_k (target_rgb) and C* (out_rgb) are float,
   IEEE binary16 or bfloat16 [3][H][W].  Values are converted to float on load
   and rounded to nearest-even on store; depth images, weights, the saved
   per-pixel state, the loss, all gradients and Adam moments stay float32. */
#define GPS_PREC_FP32 0
#define GPS_PREC_FP16 1
#define GPS_PREC_BF16 2

/* work schedule of the second pass (GpsRenderSettings.schedule) */
#define GPS_SCHEDULE_TILES 0        /* tile lists; tile-parallel backward                    */
#define GPS_SCHEDULE_PER_GAUSSIAN 1 /* OIT only, the paper's sort-free form (Sec. 3.1,
                                       App. B): unsorted tile lists for the forward (no
                                       depth cut), and a backward with one warp per
                                       Gaussian walking its pixel rectangle in groups of
                                       32 pixels; no atomics, deterministic            */

/* stage mask (GpsRenderSettings.stages; 0 = all).  Tests use it to run one
   stage on inputs they wrote into the workspace themselves. */
#define GPS_STAGE_PROJECT 1        /* records from Gaussian parameters       */
#define GPS_STAGE_BIN 2            /* tile lists from records                */
#define GPS_STAGE_COMPOSITE 4      /* forward composite (+ fused loss)       */
#define GPS_STAGE_COMPOSITE_BWD 8  /* per-Gaussian 2D gradients              */
#define GPS_STAGE_PROJECT_BWD 16   /* 2D gradients -> parameter gradients    */

/* ---------------------------------------------------------------- types */
typedef struct GpsIntrinsics {
  float fx, fy, cx, cy;
  int32_t width, height;
} GpsIntrinsics;

typedef struct GpsPose {
  float R[9]; /* camera -> world rotation, row-major */
  float t[3]; /* camera centre in world coordinates  */
} GpsPose;

/* Dense colourised TSDF (Sec. 3.1: every voxel stores d(p) and c(p)).
 * nx, ny, nz must be positive multiples of 8 (fuse_frame: ny, nz at most
 * 8 * 65535).  Voxel (x, y, z) has its centre
 * at origin + (x + 0.5, y + 0.5, z + 0.5) * voxel and is stored at the
 * brick-major index
 *     ((bz * (ny/8) + by) * (nx/8) + bx) * 512 + (z%8) * 64 + (y%8) * 8 + (x%8),
 * (bx, by, bz) = (x/8, y/8, z/8), in three arrays:
 *     sdf    float [n]    truncated signed distance / trunc, in [-1, 1]
 *     weight float [n]    fusion weight (0 = never observed)
 *     rgbw   float [n][4] colour (r, g, b) and its own weight.
 * A fresh volume is sdf = 1, weight = 0, rgbw = 0 (caller-initialised).
 * brick_flags (nullable) holds one byte per brick, in brick order: nonzero
 * where some voxel of the brick may hold sdf != 1.  fuse_frame sets them;
 * raycast_sdf then skips the voxel loads of every trilinear sample whose
 * bricks are all clear (the sample is 1 there; the march is unchanged).  A
 * fresh volume has all flags clear; a caller that writes sdf itself calls
 * tsdf_mark_bricks afterwards, or passes NULL. */
typedef struct GpsTsdf {
  int32_t nx, ny, nz;
  float voxel;      /* edge length in metres           */
  float origin[3];  /* world position of the grid corner */
  float trunc;      /* truncation distance mu, metres  */
  float max_weight; /* weight cap (e.g. 100)           */
  float* sdf;
  float* weight;
  float* rgbw;
  uint8_t* brick_flags;
} GpsTsdf;

/* A Gaussian set, or a gradient / moment buffer of the same shape (a
 * buffer's sh_degree must equal the set's). */
typedef struct GpsGaussians {
  float* means;          /* [M][3] */
  float* log_scales;     /* [M][3] */
  float* quats;          /* [M][4] w, x, y, z */
  float* opacity_logits; /* [M]    */
  float* rgb;            /* [M][3] */
  int32_t M;
  int32_t sh_degree;     /* 0..3: degree of the view-dependent colour terms     */
  float* sh_rest;        /* [M][(sh_degree+1)^2 - 1][3]; NULL when sh_degree = 0 */
} GpsGaussians;

/* One view of the second rendering pass.  Inputs are device images of this
 * view's size; outputs are nullable device images written by render_forward. */
typedef struct GpsView {
  GpsIntrinsics K;
  GpsPose T_wc;
  const void* sdf_rgb;       /* C_t [3][H][W] from raycast_sdf (required);
                                element type per settings.precision            */
  const float* sdf_depth;    /* D_t [H][W]    from raycast_sdf (required)      */
  const void* target_rgb;    /* C_k [3][H][W] observed colour; nullable;
                                element type per settings.precision            */
  const float* target_depth; /* D_k [H][W]    observed depth; nullable         */
  void* out_rgb;             /* C* [3][H][W]; nullable; element type per
                                settings.precision (the loss uses C* before
                                this rounding)                                 */
  float* out_depth;          /* D* [H][W];    nullable                          */
  float* out_weight;         /* W_G [H][W] (ALPHA: 1 - T_end); nullable         */
  const float* grad_rgb;     /* dL/dC* [3][H][W] for render_backward; nullable  */
  const float* grad_depth;   /* dL/dD* [H][W]   for render_backward; nullable  */
} GpsView;

typedef struct GpsRenderSettings {
  float eps_depth;       /* epsilon of Eq. 1-2 (metres), e.g. 0.01            */
  float lambda_depth;    /* weight of the depth L1 term (0 = colour only)      */
  float near_plane;      /* Gaussians with camera z <= near are culled (0.2)  */
  int32_t blend_mode;    /* GPS_BLEND_*                                        */
  int32_t precision;     /* GPS_PREC_*: element type of the colour images      */
  int32_t tile_w, tile_h;/* pixels per tile; 0, 0 = 16 x 8; supported: 16x16,
                            16x8, 8x8, 32x8 (gps_autotune_tiles picks one)   */
  int32_t deterministic; /* 1: bitwise reproducible, also across batching of
                            views: OIT tile lists in ascending Gaussian index
                            (fixed-order emission, views of <= 6144 tiles)
                            or sorted by (depth, index) (larger views, and the
                            alpha blend); gradient sums in 64-bit fixed point
                            (OIT) or in fixed order (alpha), no float
                            atomics.  0 (OIT): lists in emission order, which
                            may change the last bits of C* run to run         */
  int32_t stages;        /* GPS_STAGE_* mask, 0 = all                          */
  int32_t instrument;    /* 1: count Gaussian-pixel evaluations (slower; for
                            measurement runs) into the view scalars           */
  int32_t schedule;      /* GPS_SCHEDULE_*                                     */
  int64_t pair_capacity; /* (super-tile, Gaussian) entries per view; 0 = 16 * M;
                            tile bins hold tiles per super-tile times as many
                            (tile, Gaussian) entries                          */
} GpsRenderSettings;

/* Adam hyper-parameters; lr per group in the order means, log_scales, quats,
 * opacity_logits, rgb (App. C: 1.6e-4, 5e-3, 1e-3, 5e-2, 2.5e-3 * 0.28209479),
 * and lr_sh_rest for the SH coefficients of degree >= 1 (App. C: 5e-4). */
typedef struct GpsAdamHyper {
  float lr[5];
  float beta1, beta2, eps;
  float lr_sh_rest;
} GpsAdamHyper;

/* Byte offsets (from the workspace base) of the regions of view `v`.  The
 * projected record of Gaussian i is 16 floats at records + 64 i:
 *   mx, my, d, sigma, conic_a, conic_b, conic_c, qmax, r, g, b, ext_x, ext_y, 0, 0, 0
 * with q = a dx^2 + 2 b dx dy + c dy^2, support {q <= qmax}, qmax =
 * 2 ln(255 sigma), and a conservative half-extent ext (ext_x < 0: culled).
 * Binning buckets Gaussians into bins with a per-bin histogram, a scan and an
 * emission, decided per view.  Where a view's lists are depth-sorted (blend
 * ALPHA; deterministic OIT views of more than 6144 tiles) the bins are
 * super-tiles of super_px x super_px pixels: each segment is sorted, then
 * split into its tiles (when a tile is a whole super-tile its list is the
 * segment itself: tile_ranges == super_ranges and pair_keys == super_keys).
 * Otherwise (tile_bins = 1, super_px = 0) the bins are the tiles themselves
 * (super_x = tiles_x, super_y = tiles_y) and the emission writes the tile
 * lists directly: tile_ranges == super_ranges, pair_keys == super_keys ==
 * super_scratch; this needs tiles_x * tiles_y <= 16384, else the view takes
 * the super-tile path.  Deterministic OIT views binned into tiles get their
 * lists in ascending Gaussian index: the histogram's per-block counts in
 * block_base become bases by a prefix over the blocks, and the emission
 * places each block's entries warp by warp.  Tile lists: keys u64 =
 * bits(d) << 32 | index, sorted ascending where depth-sorted, by index in
 * deterministic mode's fixed order, else in emission order; tile t's list is
 * pair_keys[tile_ranges[t][0] .. tile_ranges[t][1]) (lists are not
 * contiguous).
 * grad2d holds 12 floats per Gaussian: d/d(mx, my, conic_a, conic_b, conic_c,
 * sigma, r, g, b, d), 0, 0. */
typedef struct GpsWorkspaceLayout {
  size_t total_bytes;
  size_t status;        /* int32 status word (shared by all views)            */
  size_t records;       /* float [M][16]                                      */
  size_t super_counts;  /* uint32 [bins]                                      */
  size_t block_base;    /* uint32 [binning CTAs][bins] (a CTA takes up to 8
                           chunks of 256 Gaussians)                           */
  size_t super_ranges;  /* uint32 [bins][2]                                   */
  size_t super_keys;    /* uint64 [pair_capacity] super-tile segments (tile
                           bins: the tile lists)                              */
  size_t super_scratch; /* uint64 [pair_capacity] (sort scratch)              */
  size_t tile_ranges;   /* uint32 [tiles][2]                                  */
  size_t pair_keys;     /* uint64 [tiles per super-tile * pair_capacity]      */
  size_t pix_state;     /* float [H*W][8] saved per-pixel forward state       */
  size_t tile_partials; /* float [tiles][4] loss partial sums                 */
  size_t view_scalars;  /* float [8]: loss, colour sum, depth sum, N_valid,
                           (bin, Gaussian) entries, the deterministic pair
                           counter, then the upstream bounds max|h|, max|sv|
                           of the fixed-point backward (from the forward's
                           loss with the fused loss, per unit dL/dloss; from
                           the upstream images otherwise); then uint64 [4] evaluation
                           counters: forward tested, forward counted, backward
                           tested, backward counted (instrument = 1)          */
  size_t grad2d;        /* float [M][12]: the composite adjoint's 2D gradients
                           per Gaussian; in deterministic mode with the OIT
                           blend they are written only by a backward call
                           without GPS_STAGE_PROJECT_BWD (with it, the
                           projection adjoint reads grad_fixed directly)      */
  size_t pair_grads;    /* float [tiles per super-tile * pair_capacity][12]
                           (deterministic mode): one slot per (tile,
                           Gaussian) pair, Gaussian-major (see pair_base)     */
  size_t pix_grad;      /* float [H*W][8] per-pixel upstream terms of the
                           per-Gaussian backward (GPS_SCHEDULE_PER_GAUSSIAN):
                           dL/dC* / N, dL/dD* / N, sum dL/d(C*, D*) (C*, D*) / N,
                           D_t + eps (or -inf if the pixel has no gradient)   */
  int32_t tiles_x, tiles_y, tile_w, tile_h, super_x, super_y;
  int32_t super_px;     /* super-tile edge in pixels (16, or 32 for 32-px-wide
                           tiles); 0 with tile bins                           */
  int32_t tile_bins;    /* 1: the bins are the tiles (unsorted lists)         */
  int64_t pair_capacity;
  size_t pair_base;     /* uint32 [M] (deterministic mode): Gaussian i's first
                           pair_grads slot; its slots follow in row-major
                           order of the tiles of its rectangle                */
  size_t tile_order;    /* int32 [tiles]: the tiles in order of decreasing
                           entry count of their bin (the tile itself, or its
                           super-tile), in buckets of half an octave; the
                           composites take their tiles in this order, longest
                           lists first                                        */
  size_t grad_fixed;    /* int64 [M][10] (deterministic mode, OIT blend,
                           tile schedule): each Gaussian's 2D gradient summed
                           as integers in units of a power-of-two quantum
                           from a bound on every addend (see composite.cu),
                           so the sum is the same in any order; pair_grads
                           and pair_base are empty in that mode              */
} GpsWorkspaceLayout;

/* ---------------------------------------------------------------- calls */

/* Last error message of the calling thread ("" if none). */
GPS_API const char* gps_last_error(void);

/* Library version string. */
GPS_API const char* gps_version(void);

/* Bytes of workspace needed by render_forward / render_backward for M Gaussians
 * and these views (only K.width / K.height of each view are read).  The same
 * workspace must be passed, unmodified between the two, to the forward and the
 * backward of one iteration. */
GPS_API int32_t gps_workspace_size(int32_t M, const GpsView* views, int32_t n_views,
                           const GpsRenderSettings* settings, size_t* bytes);

/* Region offsets of view `view` inside such a workspace (for inspection and tests). */
GPS_API int32_t gps_workspace_layout(int32_t M, const GpsView* views, int32_t n_views,
                             const GpsRenderSettings* settings, int32_t view,
                             GpsWorkspaceLayout* out);

/* Copy the workspace status word to *status (synchronises `stream`).
 * Returns GPS_OK if the copy succeeded; *status holds the device-side code. */
GPS_API int32_t gps_query_status(const void* ws, size_t ws_bytes, int32_t* status, void* stream);

/* Fuse one RGB-D frame into the TSDF (Sec. 3.2.1 "SDF fusion", KinectFusion /
 * InfiniTAM rule).  For every voxel centre with camera depth z > 0 projecting
 * to the nearest pixel floor(u + 0.5), floor(v + 0.5) inside the image with
 * depth D > 0: eta = D - z; if eta >= -trunc, sdf <- (w sdf + min(1, eta/trunc))
 * / (w + 1), w <- min(w + 1, max_weight); if |eta| < trunc the colour is
 * averaged with its own weight likewise.  depth [H][W], rgb [3][H][W] are
 * device images of size K.  In-place on vol. */
GPS_API int32_t fuse_frame(GpsTsdf* vol, const float* depth, const float* rgb, const GpsIntrinsics* K,
                   const GpsPose* T_wc, void* stream);

/* Recompute vol->brick_flags from vol->sdf (flag = some voxel != 1). */
GPS_API int32_t tsdf_mark_bricks(GpsTsdf* vol, void* stream);

/* Ray-cast the TSDF (Sec. 3.1 first pass).  Per pixel, march the ray from
 * max(near, entry into the voxel-centre box) to min(far, exit) (far <= 0: exit)
 * with step max(min(f, 1) trunc, voxel / 2) on the trilinear sdf f; at the first
 * f_a > 0 >= f_b refine by the secant; D_t = camera z of the hit V^g, C_t = the
 * trilinear colour of the 8 neighbouring voxels.  No hit: 0.  Outputs:
 * out_rgb [3][H][W] of element type rgb_precision (GPS_PREC_*, rounded to
 * nearest-even from the float result), out_depth [H][W], out_vertex [H][W][3]
 * world (nullable). */
GPS_API int32_t raycast_sdf(const GpsTsdf* vol, const GpsIntrinsics* K, const GpsPose* T_wc,
                    float near_plane, float far_plane, void* out_rgb, int32_t rgb_precision,
                    float* out_depth, float* out_vertex, void* stream);

/* Second rendering pass and blend (Eq. 1-4, or Table 7's sorted variant) for
 * n_views views, and, when every view has target_rgb and target_depth, the
 * fused L1 loss (Eq. 6) written to *loss (device float, nullable):
 *   L = sum_v [ sum |C* - C_k| / (3 N_v) + lambda_depth sum |D* - D_k| / N_v ]
 * over pixels with D_k > 0 and D_t > 0 (N_v of them).  Writes the views'
 * non-null outputs and the state render_backward needs into the workspace.
 * The OIT blend is order-independent, so it runs sort-free: each tile's list
 * keeps the order of the binning's emission (in deterministic mode a fixed
 * order, ascending index; depth-sorted for views of more than 6144 tiles)
 * and every warp skips the Gaussians behind all of its pixels.  The "with
 * sort" blend always sorts by (depth, index). */
GPS_API int32_t render_forward(const GpsGaussians* gaussians, const GpsView* views, int32_t n_views,
                       const GpsRenderSettings* settings, void* ws, size_t ws_bytes,
                       float* loss, void* stream);

/* Adjoint of render_forward: accumulates (+=) dL/d(parameters) into `grads`.
 * Upstream gradients: each view's grad_rgb / grad_depth if given, else the
 * derivative of the fused L1 loss (sign(C* - C_k) / (3 N_v), ...) scaled by
 * *dloss (device float; NULL = 1).  Needs the workspace of the matching
 * forward call with the same arguments. */
GPS_API int32_t render_backward(const GpsGaussians* gaussians, const GpsView* views, int32_t n_views,
                        const GpsRenderSettings* settings, void* ws, size_t ws_bytes,
                        const float* dloss, GpsGaussians* grads, void* stream);

/* Adam step (App. C learning rates, torch.optim.Adam semantics) on all five
 * groups; grads are zeroed in the same pass.  step is the 1-based step number;
 * if step <= 0 the step number is read from *device_step (int32, device),
 * incremented first, so a captured graph can replay it. */
GPS_API int32_t adam_step(GpsGaussians* params, GpsGaussians* grads, GpsGaussians* m, GpsGaussians* v,
                  const GpsAdamHyper* hyper, int32_t step, int32_t* device_step, void* stream);

/* render_backward followed by adam_step in one call, for up to 8 views: the
 * composite adjoint runs as in render_backward, then one kernel takes each
 * Gaussian's projection adjoint (summed over the views) straight into its
 * Adam update, so no parameter-gradient array is written or read.  The result
 * equals render_backward into zeroed grads followed by adam_step with the
 * same hyper-parameters and step (the same FP32 operations); `gaussians` is
 * updated in place, m and v as in adam_step.  settings.stages: 0 (all), or
 * a set holding GPS_STAGE_PROJECT_BWD (GPS_STAGE_COMPOSITE_BWD optional).
 * Errors: GPS_ERR_INVALID_ARG for more than 8 views, stages without
 * GPS_STAGE_PROJECT_BWD, and the argument errors of render_backward and
 * adam_step. */
GPS_API int32_t render_backward_adam(GpsGaussians* gaussians, const GpsView* views, int32_t n_views,
                             const GpsRenderSettings* settings, void* ws, size_t ws_bytes,
                             const float* dloss, GpsGaussians* m, GpsGaussians* v,
                             const GpsAdamHyper* hyper, int32_t step, int32_t* device_step,
                             void* stream);

/* Number of tile shapes gps_autotune_tiles tries, in this order:
 * 16x16, 16x8, 8x8, 32x8 (pixels; the binning split and both composite kernels
 * run one thread per tile pixel, so this also picks their CTA shape). */
#define GPS_AUTOTUNE_SHAPES 4

/* Tile-shape autotuner (the paper has no counterpart).  For every shape above
 * whose workspace (gps_workspace_size) fits in ws_bytes, runs render_forward +
 * render_backward on the caller's own Gaussians and views once untimed, then
 * times every shape once per round for `repeats` rounds (at most 64) with
 * CUDA events on `stream`, and returns the shape of the lowest median in
 * *best_tile_w, *best_tile_h; times_ms[GPS_AUTOTUNE_SHAPES] (nullable)
 * receives each shape's median milliseconds per forward + backward, -1 for a
 * shape that was skipped (workspace too small, or the pair capacity
 * overflowed).  settings supplies everything but the tile (stages and
 * instrument are ignored).  The backward accumulates into scratch_grads (same
 * shape as the Gaussians), which the caller discards; the views' outputs
 * are overwritten.  Synchronises `stream` after every timed pass: call it before
 * capturing graphs, then pass the chosen shape in GpsRenderSettings (and size
 * the workspace for it).  Errors: GPS_ERR_INVALID_ARG for NULL arguments,
 * render_forward's and render_backward's own errors, GPS_ERR_WORKSPACE_TOO_SMALL
 * when no shape could run. */
GPS_API int32_t gps_autotune_tiles(const GpsGaussians* gaussians, const GpsView* views,
                                   int32_t n_views, const GpsRenderSettings* settings, void* ws,
                                   size_t ws_bytes, GpsGaussians* scratch_grads, int32_t repeats,
                                   int32_t* best_tile_w, int32_t* best_tile_h, float* times_ms,
                                   void* stream);

/* ------------------------------------------ Gaussian insertion and removal */

/* Thresholds of Sec. 3.2 (defaults in brackets are the paper's). */
typedef struct GpsEditSettings {
  float delta_c;          /* insertion: mean |C* - C_k| over the channels above [0.05] */
  float delta_w;          /* insertion: Gaussian weight W_G below [4]             */
  float sample_fraction;  /* insertion: share of the mask pixels sampled [0.25]   */
  int32_t radius;         /* insertion: half-size of the neighbour window used for
                             the disc radius, pixels [3]; at most 16           */
  uint64_t seed;          /* insertion: SplitMix64 seed of the sampling draw      */
  float delta_sigma;      /* removal: opacity below [0.005]                       */
  float delta_smax;       /* removal: largest scale above [0.1] (metres)          */
  float delta_smin;       /* removal: largest scale below [0.003]                 */
  int32_t precision;      /* GPS_PREC_* of rendered_rgb and target_rgb            */
} GpsEditSettings;

/* Scratch bytes insert_gaussians / remove_gaussians need for `capacity`
 * Gaussians and width x height images (caller-allocated, 256-byte aligned). */
GPS_API int32_t gps_edit_scratch_size(int32_t capacity, int32_t width, int32_t height,
                                      size_t* bytes);

/* Gaussian insertion (Sec. 3.2 "Gaussian insertion", App. A) for one frame.
 * The mask holds the pixels the ray-cast hit (sdf_depth > 0) whose colour
 * error, taken in float32 as (|e_r| + |e_g|) + |e_b| > float(3 delta_c) with
 * e = C* - C_k, is above delta_c and whose Gaussian weight is below delta_w.
 * A pixel p (row-major) is sampled when it is in the mask and the top 24 bits
 * of the (p + 1)-th output of SplitMix64 seeded with `seed` are below
 * sample_fraction * 2^24.  Each sampled pixel u, in pixel order, appends one
 * Gaussian at index M, M + 1, ... (up to `capacity`): mean = vertex(u),
 * rgb = C_k(u), opacity logit 0 (sigma = 0.5), a flat disc with scales
 * (s1, s1, 0.1 s1), s1 = min(0.1, sqrt of the mean squared distance from
 * vertex(u) to the (at most) three nearest vertices of mask pixels within
 * `radius` pixels; none: depth(u) / fx), whose short axis is the vertex-map
 * normal at u turned to face the camera.  The new rows of m, v and grads
 * (each nullable) are zeroed.
 *   gaussians: arrays of `capacity` rows, gaussians->M = the current count.
 *   vertex [H][W][3] world points from raycast_sdf; sdf_depth, weight [H][W]
 *   float; rendered_rgb (C*) and target_rgb (C_k) [3][H][W] of type
 *   s->precision; all device memory of the size K gives.
 *   *count (device int32) receives the new count min(M + sampled, capacity).
 * Enqueued on `stream`, no synchronisation; errors: GPS_ERR_INVALID_ARG,
 * GPS_ERR_WORKSPACE_TOO_SMALL (scratch), GPS_ERR_CUDA. */
GPS_API int32_t insert_gaussians(GpsGaussians* gaussians, int32_t capacity, GpsGaussians* m,
                                 GpsGaussians* v, GpsGaussians* grads, const GpsIntrinsics* K,
                                 const GpsPose* T_wc, const float* vertex, const float* sdf_depth,
                                 const void* rendered_rgb, const float* weight,
                                 const void* target_rgb, const GpsEditSettings* s, void* scratch,
                                 size_t scratch_bytes, int32_t* count, void* stream);

/* Gaussian removal (Sec. 3.2 "Gaussian removal"): deletes the Gaussians of
 * [0, gaussians->M) with opacity logit < float(ln(delta_sigma / (1 - delta_sigma)))
 * or largest log-scale > float(ln delta_smax) or < float(ln delta_smin), and
 * compacts the rest to [0, kept) in their order, together with the same rows
 * of m, v and grads (nullable; rows [kept, M) of those are zeroed).  *count
 * (device int32) receives kept.  Enqueued on `stream`; errors as above. */
GPS_API int32_t remove_gaussians(GpsGaussians* gaussians, GpsGaussians* m, GpsGaussians* v,
                                 GpsGaussians* grads, const GpsEditSettings* s, void* scratch,
                                 size_t scratch_bytes, int32_t* count, void* stream);

/* ------------------------------------------------------------ voxel hashing
 * The TSDF of Sec. 3.2.1 kept in a hash table of voxel blocks, as InfiniTAM
 * keeps it: 8^3-voxel bricks (x fastest inside, as in GpsTsdf) live in a pool
 * of `capacity` bricks and are found through an open-addressing table keyed
 * by the brick's linear index bx + nbx (by + nby bz) in an nx x ny x nz grid,
 * which may be far larger than the pool.  A brick is allocated at the start
 * of the frame in which one of its voxels first lies within the truncation
 * band (|eta| < trunc, with fuse_frame's projection, pixel and arithmetic);
 * from then on every fused frame updates its voxels by fuse_frame's rule.
 * Bricks never allocated read as sdf 1, colour 0.  No brick is freed.
 * The caller allocates every array and zeroes `keys` and `state` for a fresh
 * volume; allocation initialises a brick's voxels (sdf 1, weights 0, colour 0).
 * Device-side failures (pool full, candidate set full, a table probe over 64
 * buckets) set state[1] to GPS_ERR_CAPACITY; the brick is then not stored. */
typedef struct GpsHashTsdf {
  int32_t nx, ny, nz;       /* index space, voxels; multiples of 8, each < 2^21  */
  float voxel;              /* edge length, metres                               */
  float origin[3];          /* world position of the grid corner                 */
  float trunc;              /* truncation distance mu, metres                    */
  float max_weight;         /* weight cap                                        */
  int32_t n_buckets;        /* hash table size, a power of two >= 2 * capacity   */
  int32_t capacity;         /* bricks in the pool                                */
  uint64_t* keys;           /* [n_buckets]: 0 = empty, else brick index + 1      */
  int32_t* slots;           /* [n_buckets]: pool slot of the bucket's brick      */
  int64_t* brick_of_slot;   /* [capacity]: brick index held by each pool slot    */
  int32_t* state;           /* [4] device: bricks in use, error code, -, -       */
  float* sdf;               /* [capacity][512]                                   */
  float* weight;            /* [capacity][512]                                   */
  float* rgbw;              /* [capacity][512][4]: colour and its weight         */
  uint8_t* slot_flags;      /* [capacity] (nullable): 1 once a voxel of the slot's
                               brick has left sdf 1 (set by fusion, 0 when the
                               brick is allocated); the ray-cast then skips the
                               loads of stored bricks whose flag is 0, with the
                               same result                                       */
} GpsHashTsdf;

/* Scratch bytes of fuse_frame_hashed for up to max_candidates candidate
 * bricks per frame (bricks within the truncation band's reach of some pixel;
 * a 640 x 480 frame of a room touches a few thousand). */
GPS_API int32_t gps_hash_scratch_size(int32_t max_candidates, size_t* bytes);

/* Fusion of one frame into the hashed volume: candidate bricks from every
 * pixel's band segment (a conservative superset), the exact band test on
 * each candidate's voxels, allocation of the bricks that pass, then
 * fuse_frame's update on every allocated brick in view.  Errors:
 * GPS_ERR_INVALID_ARG for NULL pointers or bad sizes,
 * GPS_ERR_WORKSPACE_TOO_SMALL for scratch below gps_hash_scratch_size;
 * capacity overflows are reported in state[1] (see above). */
GPS_API int32_t fuse_frame_hashed(GpsHashTsdf* vol, const float* depth, const float* rgb,
                                  const GpsIntrinsics* K, const GpsPose* T_wc, void* scratch,
                                  size_t scratch_bytes, int32_t max_candidates, void* stream);

/* raycast_sdf on the hashed volume (same march, same outputs; bricks not
 * allocated are empty space). */
GPS_API int32_t raycast_sdf_hashed(const GpsHashTsdf* vol, const GpsIntrinsics* K,
                                   const GpsPose* T_wc, float near_plane, float far_plane,
                                   void* out_rgb, int32_t rgb_precision, float* out_depth,
                                   float* out_vertex, void* stream);

/* Copies every allocated brick into the dense volume `dense` (same nx, ny,
 * nz, brick-major layout) and sets its brick flag when a voxel's sdf differs
 * from 1; the rest of `dense` is left as it is (initialise it as a fresh
 * volume first).  For inspection and tests. */
GPS_API int32_t tsdf_hash_to_dense(const GpsHashTsdf* vol, GpsTsdf* dense, void* stream);

/* ------------------------------------------------------------ camera tracking
 * Point-to-plane ICP (Sec. 3.2 "Camera tracking", Eq. 5, after KinectFusion
 * and InfiniTAM).  Gauss-Newton over a depth pyramid, coarsest level first;
 * one iteration at one level:
 *   1. p = T V_k(u) for every pixel u of the level with a depth and a normal
 *      (V_k: the level's camera-frame vertex map, T the current estimate);
 *   2. u^ = the nearest pixel, floor(x + 0.5), of p projected into the
 *      reference view (intrinsics K, pose T_ref, full resolution);
 *   3. u counts when u^ is inside, the reference has a hit and a normal
 *      there, |p - V*(u^)| < eps_d and the angle between R N_k(u) and
 *      N*(u^) is below eps_theta;
 *   4. r = (p - V*(u^)) . N*(u^), J = [N*^T, (p x N*)^T];
 *   5. xi = -(sum J^T J)^-1 sum J^T r (Cholesky, single precision), and
 *      T <- exp(xi^) T with xi = (translation, rotation); a system that is
 *      not positive definite leaves T unchanged.
 * Level l + 1 holds the mean of the valid depths of each 2x2 block of level
 * l, with intrinsics f / 2, c / 2 (coarse pixel i on fine pixel 2i).  Normals (current levels and
 * reference) are the cross product of central differences, (V(x+1) - V(x-1))
 * x (V(y+1) - V(y-1)), turned towards the camera; a pixel lacking one of its
 * four neighbours has none. */
typedef struct GpsIcpSettings {
  int32_t levels;       /* pyramid levels [3], 1..4                             */
  int32_t iters[4];     /* iterations per level, finest first [10, 5, 4, 0]     */
  float eps_d;          /* association distance, metres [0.1]                   */
  float eps_theta_deg;  /* association normal angle, degrees [20]              */
} GpsIcpSettings;

/* Workspace bytes icp_track needs for width x height frames. */
GPS_API int32_t gps_icp_workspace_size(int32_t width, int32_t height, const GpsIcpSettings* s,
                                       size_t* bytes);

/* Tracks one frame.  depth [H][W] (metres, 0 = none): the current frame;
 * ref_vertex [H][W][3] (world) and ref_depth [H][W] (> 0 where the ray hit):
 * raycast_sdf's vertex and depth outputs at pose T_ref; pose (device float
 * [12], R row-major then t, camera->world): the initial estimate on entry,
 * the result on exit; stats (device float [sum of iters][2], nullable): per
 * iteration the inlier count and sum r^2 before its update.  Everything runs
 * on `stream` with no host synchronisation (graph capturable).  Errors:
 * GPS_ERR_INVALID_ARG for NULL pointers, bad sizes or settings (levels
 * outside 1..4, a level smaller than 3 x 3, negative iterations, non-positive
 * thresholds), GPS_ERR_WORKSPACE_TOO_SMALL. */
GPS_API int32_t icp_track(const GpsIntrinsics* K, const float* depth, const float* ref_vertex,
                          const float* ref_depth, const GpsPose* T_ref,
                          const GpsIcpSettings* s, float* pose, void* ws, size_t ws_bytes,
                          float* stats, void* stream);

/* ------------------------------------------- keyframes and optimisation views
 * Host-only bookkeeping of the online loop (Sec. 3.2 "Gaussian optimization",
 * Fig. 5, App. C): which frames become keyframes, and which frames one
 * Gaussian optimisation renders.  These calls touch no device memory and
 * launch nothing; they are deterministic functions of their arguments. */
typedef struct GpsViewSchedule {
  float delta_angle_deg; /* keyframe when the rotation from the last keyframe
                            exceeds this many degrees [30] (App. C)          */
  float delta_move;      /* ... or the camera centre moved more than this,
                            metres [0.3] (App. C)                            */
  int32_t interval;      /* delta_k: frames between optimisations [10]       */
  int32_t n_global;      /* keyframes drawn from the history [4], <= 1024    */
  int32_t n_local;       /* frames spread over the last interval [4]         */
  int32_t reserved;      /* 0                                                */
  uint64_t seed;         /* SplitMix64 seed of the keyframe draw             */
} GpsViewSchedule;

/* *is_keyframe = 1 when last_keyframe is NULL (the first frame), or when the
 * relative pose last_keyframe^-1 * T_wc rotates by more than delta_angle_deg
 * (angle of R_last^T R from its trace) or moves the camera centre by more
 * than delta_move (both strict), else 0.  Evaluated in double precision.
 * Errors: GPS_ERR_INVALID_ARG for NULL T_wc / s / is_keyframe or a
 * non-finite threshold. */
GPS_API int32_t gps_is_keyframe(const GpsPose* last_keyframe, const GpsPose* T_wc,
                                const GpsViewSchedule* s, int32_t* is_keyframe);

/* Views of the optimisation number `event` (0, 1, ...) taken at frame
 * `frame` (Fig. 5).  Writes to views[0 .. *n_views):
 *   1. n = min(n_local, L) local frames, L = min(interval, frame + 1):
 *      frame - floor(j L / n) for j = 0 .. n - 1 (newest first);
 *   2. min(n_global, H) keyframes drawn uniformly without replacement from
 *      the H entries of `keyframes` (ascending frame ids, n_keyframes of them)
 *      that are <= frame - interval: a partial Fisher-Yates shuffle whose
 *      step i swaps position i with i + floor(hi32(r) (H - i) / 2^32), r the
 *      (1024 event + i + 1)-th output of SplitMix64 seeded with s->seed;
 *      written in draw order.
 * Errors: GPS_ERR_INVALID_ARG for NULL pointers (keyframes may be NULL when
 * n_keyframes is 0), frame < 0, event < 0, interval < 1, n_local < 0,
 * n_global outside [0, 1024], keyframe ids not strictly ascending or
 * negative, or capacity below the number of views. */
GPS_API int32_t gps_select_views(const int32_t* keyframes, int32_t n_keyframes, int32_t frame,
                                 int32_t event, const GpsViewSchedule* s, int32_t* views,
                                 int32_t capacity, int32_t* n_views);

/* Size of the static device array behind render_forward_noalloc: 64 MiB,
 * held by every GPU that loads this library until the process exits. */
#define GPS_NOALLOC_SCRATCH_BYTES (64u << 20)

/* render_forward without a caller-provided workspace.  The paper has no
 * counterpart: this entry point exists for callers that may not call
 * cudaMalloc - for example code running inside a host application that owns
 * every device allocation (a plug-in), or a real-time loop whose device memory
 * is fixed at start-up.  It runs the full forward (settings.stages is ignored)
 * on a file-scope static device array of GPS_NOALLOC_SCRATCH_BYTES and
 * allocates nothing: no cudaMalloc, no cudaFree, no allocating library call.
 *   - Arguments, outputs (views' out_* images, *loss) and errors are those of
 *     render_forward; a problem whose workspace (gps_workspace_size) exceeds
 *     GPS_NOALLOC_SCRATCH_BYTES is rejected with GPS_ERR_WORKSPACE_TOO_SMALL
 *     before anything is launched.
 *   - The first call on each device performs a one-time set-up with that
 *     device current (it looks up the array's device address with
 *     cudaGetSymbolAddress); make that first call before any stream capture
 *     begins.
 *   - Every call on a device shares the one array, and the array keeps the
 *     last call's contents (so render_backward cannot be paired with it):
 *     calls whose work overlaps on the GPU - on different streams or from
 *     different threads - race with each other and must be serialised by the
 *     caller.
 *   - Errors found on the device (a pair-capacity overflow) land in the
 *     array's status word: read it with gps_noalloc_query_status.
 *   - The array's device address is cached per device for the life of the
 *     process; a cudaDeviceReset (or any reset of the device's primary
 *     context) invalidates it, so call neither while this library is in use. */
GPS_API int32_t render_forward_noalloc(const GpsGaussians* gaussians, const GpsView* views,
                                       int32_t n_views, const GpsRenderSettings* settings,
                                       float* loss, void* stream);

/* The status word of the static array behind render_forward_noalloc on the
 * current device, as gps_query_status reads a workspace's: *status receives
 * GPS_OK or the device-side code of the last call (GPS_ERR_CAPACITY when its
 * (tile, Gaussian) pairs overflowed settings.pair_capacity and the render is
 * truncated).  Synchronises `stream`; does the one-time set-up of
 * render_forward_noalloc if it has not run on this device.  No counterpart in
 * the paper. */
GPS_API int32_t gps_noalloc_query_status(int32_t* status, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GPS_H_ */
