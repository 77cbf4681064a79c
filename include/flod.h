/*
 * flod.h -- C ABI of the GB300 (sm_103a) splatting path of FLoD
 * ("FLoD: Integrating Flexible Level of Detail into 3D Gaussian Splatting for
 * Customizable Rendering", arXiv 2408.12894).
 *
 * The path renders and differentiates one level of a multi-level 3D Gaussian set, or a
 * distance-selected mix of levels, through a tile-based rasterizer:
 *
 *   flod_select_levels   Eq. 6 / Eq. 7 (Sec. 5.2): per-Gaussian level band by distance
 *   flod_preprocess      Eq. 4 (Sec. 4.1) scale constraint, Eq. 1 (Sec. 3) covariance,
 *                        projection to 2D (Eq. 2, Sec. 3), SH colour, extent, tile rect
 *   flod_bin_sort        (tile, depth) keys and their stable radix sort; tile ranges
 *   flod_render_fwd      depth-ordered alpha blending (Sec. 3, after Eq. 2)
 *   flod_render_bwd      gradient of the above to means, s_opt, quaternions, opacity
 *                        logits and SH (the Backpropagation step of Algorithm 1)
 *   flod_adjust_scale    Eq. 5 (Sec. 4.2, AdjustScale of Algorithm 1)
 *
 * Conventions shared by every call
 * --------------------------------
 * - All array pointers are DEVICE pointers of the current CUDA device, allocated by the
 *   caller; the library never allocates device memory and keeps no state between calls
 *   except a per-device cache of occupancy figures.
 * - Calls enqueue work on `stream` and return without waiting. Argument checks are done on
 *   the host before anything is enqueued; on a check failure nothing is enqueued and the
 *   status says why. Errors found on the device (pair capacity exceeded, inconsistent
 *   per-unit tile counts) set bits of the workspace status word, read with
 *   flod_read_status().
 *   No call aborts, traps or prints.
 * - Cameras: world->camera [R|t] row-major 3x4 (OpenCV axes: x right, y down, z forward),
 *   pinhole u = fx*x/z + cx, v = fy*y/z + cy; pixel (i, j) samples at (i+0.5, j+0.5).
 * - Gaussians are structure-of-arrays float32: means [n,3], quats [n,4] (w,x,y,z, any
 *   nonzero length), s_opt [n,3] (the learnable scale of Eq. 4), opacity_logit [n]
 *   (opacity = sigmoid), sh [n,(deg+1)^2,3] (real SH, Condon-Shortley phase, index
 *   l*l+l+m; colour = max(0, sum + 0.5)).
 * - A "view" is one camera rendering one source of Gaussians: a whole set, or a selection
 *   list from flod_select_levels. Several views in one call form a batch: every stage runs
 *   once over all views (one launch per kernel) and the per-view outputs are concatenated.
 */
#ifndef FLOD_H
#define FLOD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *flod_stream; /* a cudaStream_t; NULL = the legacy stream */

typedef enum {
  FLOD_OK = 0,
  FLOD_ERR_INVALID_ARG = 1, /* a pointer, size or enum out of range; nothing enqueued */
  FLOD_ERR_CAPACITY = 2,    /* more (Gaussian, tile) pairs than pair_capacity */
  FLOD_ERR_TIMEOUT = 3,     /* a bounded device-side wait ran out */
  FLOD_ERR_CUDA = 4,        /* a CUDA runtime call failed (launch, memset) */
  FLOD_ERR_UNSUPPORTED = 5, /* e.g. no sm_103a device */
  FLOD_ERR_WORKSPACE = 6    /* workspace smaller than flod_workspace_size() */
} flod_status;

/* Device status bits (flod_read_status). */
#define FLOD_DEV_CAPACITY 0x1u /* pairs exceeded pair_capacity: pairs beyond it dropped */
#define FLOD_DEV_TIMEOUT 0x2u  /* reserved for a bounded device-side wait that gave up; no
                                  kernel of this library spins on a flag (its only waits are
                                  barriers among the threads of one CTA), so none sets it */
#define FLOD_DEV_TILESET 0x4u  /* emission listed another tile count than tiles_touched
                                  (only with inconsistent per-unit inputs in the workspace) */
#define FLOD_DEV_GRID 0x8u     /* flod_overlap_prune: the set spans more than 2^21 cells of
                                  3 d_OP on an axis; nothing was pruned */
#define FLOD_DEV_SELECTION 0x10u /* flod_preprocess: a view's *sel_count exceeded its
                                    sel_capacity; the entries past the capacity were not
                                    rendered (grow the selection buffer and the view) */

#define FLOD_MAX_VIEWS 128
#define FLOD_MAX_SETS 16
#define FLOD_SEL_SHIFT 28 /* selection entry = (set << FLOD_SEL_SHIFT) | index */
#define FLOD_MAX_PAIRS ((1ull << 32) - 8192)

typedef struct {
  float viewmat[12]; /* world -> camera, row-major [R | t] */
  float fx, fy, cx, cy;
  int width, height;
  float cam_pos[3]; /* camera centre in world space (SH view direction) */
} flod_camera;

typedef struct {
  const float *means;
  const float *quats;
  const float *s_opt;
  const float *opacity_logit;
  const float *sh;
  int n;         /* Gaussians in the set, < 2^28 */
  int sh_degree; /* 0..3 */
  float s_min;   /* the level's 3D scale constraint s_min^(l) of Eq. 3/4 */
} flod_gaussians;

typedef struct {
  flod_camera cam;
  int set;                    /* index into the `sets` array when sel == NULL */
  const uint32_t *sel;        /* optional selection entries (set << 28) | index */
  const uint32_t *sel_count;  /* device count of valid entries of sel (with sel) */
  uint32_t sel_capacity;      /* entries reserved for sel (the units of this view; a
                                 *sel_count above it renders the first sel_capacity entries
                                 and sets FLOD_DEV_SELECTION) */
} flod_view;

typedef struct {
  int tile_w, tile_h; /* 8x8, 16x16 or 32x8 pixels */
  int batch;          /* Gaussians staged per shared-memory batch: 32, 64, 128 or 256 (the
                         blending kernels stage at most 128) */
  float dilation;     /* px^2 added to the 2D covariance diagonal (default 0.3) */
  float z_near;       /* cull t_z <= z_near (default 0.2) */
  float bg[3];        /* background colour (default black) */
  int extent_rule;    /* 2 (default): opacity-aware support ellipse, listed row by row
                         (tile columns whose pixel centres meet it); 0: its bounding circle's
                         square; 1: 3 sigma square */
  int persistent;     /* 1: flod_bin_sort also orders the tiles largest-first (by pair
                         count) and the renderers run persistent CTAs over that order */
} flod_raster_config;

/* Gradient outputs of one set, same shapes as the parameters (quats and, at SH degree 3,
 * sh 16-byte aligned). `overwrite` selects how they are written:
 *   0  accumulated with += into the caller's values;
 *   1  every gradient of the set is written once (zeros for Gaussians that touch no tile),
 *      which needs no zeroed buffers; requires that exactly one view renders the set, as a
 *      whole set (no selection list), else the call returns FLOD_ERR_INVALID_ARG;
 *   2  the library zero-fills the set's buffers (one kernel in the call's stream, before the
 *      gradients are added), then accumulates as with 0: any views, no caller fill needed.
 * Other values return FLOD_ERR_INVALID_ARG. */
typedef struct {
  float *means, *quats, *s_opt, *opacity_logit, *sh;
  int overwrite;
} flod_grads;

/* Byte offsets of the workspace's regions (see flod_workspace_layout). */
typedef struct {
  size_t total;         /* bytes required */
  size_t status;        /* uint32 status bits */
  size_t pair_count;    /* uint64 pairs emitted by the last flod_bin_sort */
  size_t plan;          /* uint32[64] radix-sort plan; plan[63] = buffer index of the result;
                           uint64 at plan[48] / plan[50]: running count of (pixel, Gaussian)
                           evaluations of the blending forward / backward kernels; at
                           plan[52]: of the pairs the forward blended */
  size_t xy;            /* float2 [units] projected mean (u, v) */
  size_t depth;         /* float [units] view-space z */
  size_t conic_o;       /* float4 [units] (a, b, c, opacity), q = a dx^2 + 2b dx dy + c dy^2 */
  size_t rgb;           /* float4 [units] (r, g, b, 0) */
  size_t radius;        /* float [units] extent radius in pixels (rules 0, 1; rule 2: the
                           rule-0 circle radius, informational) */
  size_t ext;           /* float4 [units] the support ellipse (alpha >= 1/255, widened by a
                           relative 2^-10) as (m, h, rx, ry): its rows are
                           x = u + m dy +- h sqrt(ry^2 - dy^2), its bounding half-widths rx,
                           ry; zero when the support is empty. Rule 2 bins by it */
  size_t trec;          /* uint4 [units] tile record written by preprocess for the emission:
                           x = tx0 | ty0 << 16 (first tile column and row), y = rows |
                           mode << 16; mode 0: z, w hold up to 4 rows of (column offset,
                           count) in 8 + 8 bits; mode 1: z = tiles per row; mode 2: rows are
                           recomputed from xy and ext */
  size_t tiles_touched; /* uint32 [units], 0 when culled */
  size_t block_sums;    /* uint64 [units/1024 + 1] exclusive pair offsets per 1024 units */
  size_t slices;        /* uint32 [units/1024 + 1] exclusive count of 4096-pair emission slices */
  size_t ukeys[2];      /* uint32 [units] x 2: depth keys of the unit-stage sort; after it,
                           ukeys[0] holds the tile count of every depth-sorted slot */
  size_t uvals[2];      /* uint32 [units] x 2: units in depth order (plan[45] = result buffer) */
  size_t keys[2];       /* uint32 [pair_capacity] x 2: tile ids of the pairs (keys[0] = emitted;
                           during emission keys[1], vals[1] list the units written by whole
                           half-warps: first position, unit) */
  size_t vals[2];       /* uint32 [pair_capacity] x 2: units of the pairs */
  size_t hist;          /* radix-sort digit histograms */
  size_t counts;        /* uint32 [512][partitions]: radix sort, per-partition digit counts */
  size_t ranges;        /* uint32x2 [tiles] [start, end) in the sorted pair list */
  size_t grad2d;        /* float [units][9]: du, dv, dopacity, da, db, dc, dr, dg, db */
  size_t queue;         /* uint32 [tiles + 128]: 66 header words, then the largest-first tile order */
  uint64_t units;       /* total units (each view's capacity rounded up to 1024) */
  uint64_t tiles;       /* total tiles over all views */
  uint64_t pixels;      /* total pixels over all views */
  uint64_t pair_capacity;
} flod_ws_layout;

/* Fill *cfg with the defaults: 16x16 tiles, batch 128, dilation 0.3, z_near 0.2, black
 * background, opacity-aware extent, one CTA per tile. */
void flod_default_config(flod_raster_config *cfg);

/* Workspace bytes for a batch of views; the pair capacity bounds the (Gaussian, tile)
 * pairs of all views together (<= FLOD_MAX_PAIRS). Returns 0 on invalid arguments. */
size_t flod_workspace_size(const flod_gaussians *sets, int n_sets, const flod_view *views,
                           int n_views, uint64_t pair_capacity, const flod_raster_config *cfg);

/* Offsets of every workspace region, plus the per-view unit, tile and pixel offsets
 * (arrays of n_views + 1 entries each, may be NULL). Pure host computation.
 * The stage calls below all take the same (sets, views, cfg, pair_capacity) description,
 * which must not change between the calls of one frame: the workspace layout is a function
 * of it alone, and ws must be 256-byte aligned and at least flod_workspace_size() bytes. */
flod_status flod_workspace_layout(const flod_gaussians *sets, int n_sets, const flod_view *views,
                                  int n_views, uint64_t pair_capacity,
                                  const flod_raster_config *cfg, flod_ws_layout *out,
                                  uint64_t *unit_offset, uint64_t *tile_offset,
                                  uint64_t *pixel_offset);

/* Eq. 4 + Eq. 1 + Eq. 2 projection + SH colour per (view, Gaussian): fills the unit
 * arrays of the workspace (xy, depth, conic_o, rgb, radius, tiles_touched) and clears the
 * status word. A unit is culled (tiles_touched = 0) when t_z <= z_near, when its 2D
 * covariance is not positive definite, when opacity < 1/255 (opacity-aware extent) or when
 * its rectangle misses the image. */
flod_status flod_preprocess(const flod_gaussians *sets, int n_sets, const flod_view *views,
                            int n_views, const flod_raster_config *cfg, void *ws,
                            size_t ws_bytes, uint64_t pair_capacity, flod_stream stream);

/* (tile, depth) binning and sort: the pairs (unit, covered tile) end up ordered by the key
 * (global tile << 32) | float bits of t_z, ties by unit index -- the stable sort of the pairs
 * emitted in unit order. It is a stable LSD radix sort (reduce-then-scan passes over
 * 4,096-key partitions; four 8-bit depth digits, tile digits of at most 9 bits) whose depth
 * digits are sorted over units before the pairs are emitted, since all pairs of a unit share
 * them, and whose tile digits are sorted over the pairs. Then the [start, end) range of every tile. The result is vals[plan[63]] (units)
 * with keys[plan[63]] (tile ids). Writes the pair total to *d_pair_count (device, may be
 * NULL) and to the workspace. Pairs beyond pair_capacity are dropped and FLOD_DEV_CAPACITY
 * is set. */
flod_status flod_bin_sort(const flod_gaussians *sets, int n_sets, const flod_view *views,
                          int n_views, const flod_raster_config *cfg, void *ws, size_t ws_bytes,
                          uint64_t pair_capacity, uint64_t *d_pair_count, flod_stream stream);

/* flod_bin_sort in parts, for callers that time them separately: phase FLOD_BIN_ALL is
 * flod_bin_sort itself; phases 1..4, called in order with the same arguments, enqueue
 * exactly the same kernels:
 *   FLOD_BIN_PHASE_DEPTH    the depth order of the units with tiles (their compaction and
 *                           the depth-digit passes; also clears the tile ranges);
 *   FLOD_BIN_PHASE_EMIT     per-block pair offsets, their scan (pair total to *d_pair_count
 *                           and the workspace) and the emission of the pairs in depth order;
 *   FLOD_BIN_PHASE_TILES    the tile-digit passes over the pairs;
 *   FLOD_BIN_PHASE_RANGES   the tile ranges (and, with cfg->persistent, the largest-first
 *                           tile order).
 * Any other phase returns FLOD_ERR_INVALID_ARG. */
#define FLOD_BIN_ALL 0
#define FLOD_BIN_PHASE_DEPTH 1
#define FLOD_BIN_PHASE_EMIT 2
#define FLOD_BIN_PHASE_TILES 3
#define FLOD_BIN_PHASE_RANGES 4
flod_status flod_bin_sort_phase(const flod_gaussians *sets, int n_sets, const flod_view *views,
                                int n_views, const flod_raster_config *cfg, void *ws,
                                size_t ws_bytes, uint64_t pair_capacity, uint64_t *d_pair_count,
                                int phase, flod_stream stream);

/* Front-to-back blending per pixel of every view. Outputs (device, planar per view, views
 * concatenated at their pixel offsets): out_rgb [3][H][W] per view, out_T [H][W] final
 * transmittance, out_ncontrib [H][W] 1-based position of the last blended Gaussian in the
 * tile's sorted list. alpha = min(0.99, o exp(-q/2)); alpha < 1/255 is skipped; blending
 * stops before the Gaussian that would take T below 1e-4. out_T and out_ncontrib are
 * needed by flod_render_bwd. */
flod_status flod_render_fwd(const flod_gaussians *sets, int n_sets, const flod_view *views,
                            int n_views, const flod_raster_config *cfg, void *ws, size_t ws_bytes,
                            uint64_t pair_capacity, float *out_rgb, float *out_T,
                            uint32_t *out_ncontrib, flod_stream stream);

/* Gradient of L = sum(dL_drgb * rgb) through blending, projection, SH, Eq. 1 and Eq. 4,
 * accumulated (+=) into grads[set] for every set that a view renders (grads has n_sets
 * entries; a NULL member skips that parameter). Re-walks every pixel back to front from
 * out_T / out_ncontrib of the forward; the workspace must still hold the forward's state.
 * Gradients go through non-atomic read-modify-write when a set is rendered by one view
 * only, else through atomics; a selection list must not repeat an entry. */
flod_status flod_render_bwd(const flod_gaussians *sets, int n_sets, const flod_view *views,
                            int n_views, const flod_raster_config *cfg, void *ws,
                            size_t ws_bytes, uint64_t pair_capacity, const float *dL_drgb,
                            const float *fwd_T,
                            const uint32_t *fwd_ncontrib, const flod_grads *grads,
                            flod_stream stream);

/* The two halves of flod_render_bwd, for callers that time or use them separately.
 * flod_blend_bwd clears the per-unit 2D gradient accumulators of the workspace and runs the
 * blending backward (per-unit dL/d(u, v, conic, opacity, rgb), see flod_ws_layout.grad2d);
 * flod_preprocess_bwd chains them to the parameters (+= into grads, as flod_render_bwd). */
flod_status flod_blend_bwd(const flod_gaussians *sets, int n_sets, const flod_view *views,
                           int n_views, const flod_raster_config *cfg, void *ws, size_t ws_bytes,
                           uint64_t pair_capacity, const float *dL_drgb, const float *fwd_T,
                           const uint32_t *fwd_ncontrib, flod_stream stream);
flod_status flod_preprocess_bwd(const flod_gaussians *sets, int n_sets, const flod_view *views,
                                int n_views, const flod_raster_config *cfg, void *ws,
                                size_t ws_bytes, uint64_t pair_capacity, const flod_grads *grads,
                                flod_stream stream);

/* ---------------------------------------------------------------------------------------
 * Training step of a level (Algorithm 1: Loss, then Adam on the gradient)
 * --------------------------------------------------------------------------------------- */

/* The five parameter arrays of one set (device, float32, shapes of flod_gaussians). */
typedef struct {
  float *means, *quats, *s_opt, *opacity_logit, *sh;
} flod_param_arrays;

/* Scratch bytes of flod_loss for n_images images of the given sizes (host arrays). */
size_t flod_loss_scratch_size(const int *widths, const int *heights, int n_images);

/* The training loss of the level (Sec. 5.1.4: the backbone's "L1 and SSIM losses"; the Loss
 * step of Algorithm 1) and its gradient, per image:
 *   L = (1 - lambda) mean|I - I_hat| + lambda (1 - mean SSIM(I, I_hat)),
 * means over the image's 3 channels and pixels; SSIM of Wang et al. with an 11 x 11 Gaussian
 * window (sigma 1.5, normalised, zero outside the image), C1 = 0.01^2, C2 = 0.03^2.
 * img, target: device, the planar layout of flod_render_fwd's out_rgb ([3][H][W] per image,
 * images concatenated; widths / heights are host arrays of n_images <= FLOD_MAX_VIEWS
 * entries). Writes dL/dimg (same layout; the gradient of each image's own loss, ready for
 * flod_render_bwd) and, when d_loss is not NULL, each image's loss to d_loss[i] (device).
 * scratch: device, flod_loss_scratch_size() bytes, 256-byte aligned, no initial contents. */
flod_status flod_loss(const float *img, const float *target, const int *widths,
                      const int *heights, int n_images, float lambda, float *d_loss,
                      float *dL_dimg, void *scratch, size_t scratch_bytes, flod_stream stream);

/* Adam hyper-parameters (Adam step of Algorithm 1). One learning rate per parameter group:
 * means, rotations, s_opt, opacity logits, SH coefficient 0 (DC) and SH coefficients 1..K-1.
 * beta1, beta2 and eps are doubles: 1 - beta and the bias corrections are formed from them in
 * double before rounding (0.999 has no float32 representation close enough for 1 - beta2).
 * d_step (device uint32) counts the steps taken: a call uses t = *d_step + 1 for the bias
 * corrections and then increments it in the stream, so a captured CUDA graph replays
 * successive steps; start it at 0. */
typedef struct {
  float lr_means, lr_quats, lr_s_opt, lr_opacity, lr_sh_dc, lr_sh_rest;
  double beta1, beta2, eps;
  uint32_t *d_step;
} flod_adam_config;

/* One Adam step of n_sets sets (one launch, one advance of the step counter), per entry:
 *   m <- beta1 m + (1 - beta1) g,   v <- beta2 v + (1 - beta2) g^2,
 *   p <- p - lr (m / (1 - beta1^t)) / (sqrt(v / (1 - beta2^t)) + eps).
 * params (updated in place), grads, m, v: host arrays of n_sets entries of device arrays;
 * set k has n[k] Gaussians at SH degree sh_degree[k] (host arrays); all five members
 * non-NULL when n[k] > 0; m and v start at zero. Returns FLOD_ERR_INVALID_ARG on NULL
 * arrays, n[k] < 0 or n_sets outside 1..FLOD_MAX_SETS. */
flod_status flod_adam_step(const flod_param_arrays *params, const flod_param_arrays *grads,
                           const flod_param_arrays *m, const flod_param_arrays *v, const int *n,
                           const int *sh_degree, int n_sets, const flod_adam_config *cfg,
                           flod_stream stream);

/* Adam state of one set for flod_preprocess_bwd_adam: where the updated parameters go
 * (`params`; may be the set's own arrays) and the moments m, v (same shapes). Every array of
 * the three, and every parameter array of the set, must be 16-byte aligned. */
typedef struct {
  flod_param_arrays params, m, v;
} flod_adam_state;

/* flod_preprocess_bwd and flod_adam_step in one pass: the chain rule of each unit from the
 * blending backward's 2D gradients to the parameters, each parameter gradient consumed at once
 * by the Adam step of that entry (the gradient is never stored). Every set must be rendered
 * by exactly one view, as a whole set (no selection list), so each Gaussian has one unit;
 * Gaussians that touch no tile take the step with g = 0, as the standalone step would. states
 * has n_sets entries. The step counter advances once per call. Else as flod_preprocess_bwd. */
flod_status flod_preprocess_bwd_adam(const flod_gaussians *sets, int n_sets,
                                     const flod_view *views, int n_views,
                                     const flod_raster_config *cfg, void *ws, size_t ws_bytes,
                                     uint64_t pair_capacity, const flod_adam_state *states,
                                     const flod_adam_config *acfg, flod_stream stream);

/* Copies selected Gaussians of one or more sets into one compact set (structure of arrays):
 * for k < min(*d_count, capacity), output Gaussian k is a copy of sets[e >> 28][e & mask]
 * with e = entries[k] (entries may be NULL: then e = k, from set 0). Uses: the predetermined
 * selective set of Sec. 5.2 (the entries of flod_select_levels from the mean training-camera
 * position) made resident on its own instead of all levels; level chunks streamed from host
 * memory (the source arrays may be pinned host memory mapped for the device: the copy then
 * reads across the CPU-GPU link); pruned or densified sets.
 * - out: device arrays with room for `capacity` Gaussians at out_sh_degree (quats and, at
 *   degree 1 or 3, sh 16-byte aligned); SH coefficients beyond a source's degree are zero.
 * - fold_s_min = 1: the source set's s_min is moved into the scale parameter,
 *   s_opt' = log(exp(s_opt) + s_min), so the output renders at s_min = 0 with each
 *   Gaussian's own Eq. 4 scale (Gaussians of several levels in one set); 0: s_opt copied.
 * - out_s_min (optional, device float [capacity]): each output Gaussian's source s_min.
 * Entries naming a missing set or index leave their output untouched. */
flod_status flod_gather(const flod_gaussians *sets, int n_sets, const uint32_t *entries,
                        const uint32_t *d_count, uint32_t capacity, const flod_param_arrays *out,
                        int out_sh_degree, int fold_s_min, float *out_s_min, flod_stream stream);

/* Density-control statistics (the Densification step of Algorithm 1; the backbone's rule):
 * after flod_blend_bwd, for every unit that touches a tile, accum[set][i] += || dL/d mean2d ||
 * with the 2D mean in normalised device coordinates (the pixel gradient times (W/2, H/2)) and
 * denom[set][i] += 1, for Gaussian i of the unit's set (atomics; several views may render
 * it). accum, denom: host arrays of n_sets device float pointers (NULL skips a set). The
 * workspace must hold the backward's per-unit gradients (call before the next blending
 * backward or preprocess of that workspace). Else as flod_blend_bwd. */
flod_status flod_densify_stats(const flod_gaussians *sets, int n_sets, const flod_view *views,
                               int n_views, const flod_raster_config *cfg, void *ws,
                               size_t ws_bytes, uint64_t pair_capacity, float *const *accum,
                               float *const *denom, flod_stream stream);

/* Scratch bytes of flod_densify for a set of n Gaussians. */
size_t flod_densify_scratch_size(int n);

/* The density-control step of a level (Densification and Pruning of Algorithm 1, with the
 * backbone's rules; the paper does not remove large Gaussians, Sec. 5.1.4). Per Gaussian,
 * in float32: g = accum / denom (0 when denom is 0); s = exp(s_opt) + s_min (Eq. 4).
 *   g >= tau and max(s) <= max_clone_scale: cloned (a copy appended);
 *   g >= tau and max(s) > max_clone_scale: split into two children with means
 *     mu + R(q) (s * eps), eps = normals[2i], normals[2i + 1] (standard-normal draws given by
 *     the caller, [2n][3]), s_opt - log 1.6 (the learnable part of the scale over 1.6), every
 *     other parameter copied; the parent is removed;
 *   sigmoid(logit) < min_opacity: removed, with its clone or children.
 * The new set, written to `out` (device arrays with room for `capacity` Gaussians; quats
 * 16-byte aligned): the Gaussians kept in place by index, then the clones, then the
 * children, two per split Gaussian. Adam moments (m_in, v_in -> m_out, v_out, all NULL or
 * all given) follow the survivors and are zero for clones and children. *d_count = the new
 * set's size (device; only the first `capacity` are written); d_counts3 (optional device
 * [3]) = kept in place, clones, split Gaussians. scratch: flod_densify_scratch_size(n) bytes. */
flod_status flod_densify(const flod_gaussians *set, const float *accum, const float *denom,
                         const float *normals, float tau, float max_clone_scale,
                         float min_opacity, const flod_param_arrays *m_in,
                         const flod_param_arrays *v_in, const flod_param_arrays *out,
                         const flod_param_arrays *m_out, const flod_param_arrays *v_out,
                         uint32_t capacity, uint32_t *d_count, uint32_t *d_counts3,
                         void *scratch, size_t scratch_bytes, flod_stream stream);

/* Scratch bytes of flod_overlap_prune for a set of n Gaussians. */
size_t flod_prune_scratch_size(int n);

/* Overlap pruning (Sec. 4.3): Gaussian i of `set` is removed when the average distance from
 * its mean to the three nearest other means of the set, d_avg = (d1 + d2 + d3) / 3, is below
 * d_op (the paper's d_OP = s_min / 2 of the level being trained). Only means within 3 d_op
 * can make d_avg < d_op, so the search is exact over a uniform grid of that cell edge; a
 * Gaussian with fewer than three others within 3 d_op is kept and its d_avg reported as
 * +inf. Distances in float32 (each difference, square and sum rounded, correctly rounded
 * square root, the mean of the three).
 * Outputs (device): keep[n] (1 kept, 0 pruned); d_avg[n] (optional); out_kept[n] (optional:
 * the kept indices in increasing order, ready as flod_gather entries of the set);
 * *d_kept_count; *d_status (optional) = FLOD_DEV_GRID when the set's bounding box spans more
 * than 2^21 cells on an axis (then every Gaussian is kept). scratch: device,
 * flod_prune_scratch_size(n) bytes, 256-byte aligned, no initial contents. */
flod_status flod_overlap_prune(const flod_gaussians *set, float d_op, uint8_t *keep, float *d_avg,
                               uint32_t *out_kept, uint32_t *d_kept_count, uint32_t *d_status,
                               void *scratch, size_t scratch_bytes, flod_stream stream);

/* Eq. 6 with the thresholds of Eq. 7. levels[0..n_levels-1] are given coarse to fine.
 * d_thresh (host array of n_levels-1 floats, descending) gives d_proj of each level but the
 * last; if NULL, d_proj = s_min * focal / gamma (Eq. 7). The last level's band ends at 0 and
 * the first level's at infinity. A Gaussian of level k is kept iff
 * d_thresh[k-1] > d >= d_thresh[k], d = ||mean - origin|| in float32. Writes the kept
 * entries (k << 28) | i to out_sel in (level, index) order and their number to *d_count
 * (device). scratch: device bytes of flod_select_scratch_size() (a count per block of 2048
 * Gaussians, then their keep bits); scratch_bytes of at least 4 (blocks + 1) hold the counts
 * alone, which gives the same result with a second evaluation of Eq. 6 in the write kernel;
 * less returns FLOD_ERR_WORKSPACE. */
size_t flod_select_scratch_size(const flod_gaussians *levels, int n_levels);
flod_status flod_select_levels(const flod_gaussians *levels, int n_levels, const float *d_thresh,
                               float gamma, float focal, const float origin[3],
                               uint32_t *out_sel, uint32_t sel_capacity, uint32_t *d_count,
                               void *scratch, size_t scratch_bytes, flod_stream stream);

/* flod_select_levels without caller-provided scratch (no counterpart in the paper: this
 * is a deployment variant). Some callers cannot allocate device memory at all: a plugin
 * running inside a host application that owns every device allocation through its own
 * pool, or a real-time loop that must not take cudaMalloc's device-wide synchronisation
 * and latency. This entry point allocates nothing: the per-block counts that
 * flod_select_levels keeps in `scratch` live instead in a fixed array of
 * FLOD_SELECT_NOALLOC_MAX_BLOCKS + 1 uint32 words (64 KiB + 4 bytes) compiled into the
 * library, which every GPU that loads the library holds until the process exits. The
 * caller still provides out_sel and d_count; arguments and results are those of
 * flod_select_levels.
 * - Limit: sum over levels of ceil(n / 2048) <= FLOD_SELECT_NOALLOC_MAX_BLOCKS (at most
 *   2^25 = 33,554,432 Gaussians over all levels); larger inputs are rejected with
 *   FLOD_ERR_INVALID_ARG before anything is enqueued.
 * - The first call on a device looks up the array's device address (with that device
 *   current) and caches it; make that first call before any stream capture.
 * - Every call on a device shares the one array and leaves its contents behind. Nothing in
 *   it needs to start at zero (each call writes every word it reads), but two calls whose
 *   work overlaps on the GPU (other streams, other threads) race on it: order them. */
#define FLOD_SELECT_NOALLOC_MAX_BLOCKS 16384
flod_status flod_select_levels_noalloc(const flod_gaussians *levels, int n_levels,
                                       const float *d_thresh, float gamma, float focal,
                                       const float origin[3], uint32_t *out_sel,
                                       uint32_t sel_capacity, uint32_t *d_count,
                                       flod_stream stream);

/* Eq. 5: s_opt <- log(exp(s_opt) + s_min_cur - s_min_next) in place, so that the scale of
 * Eq. 4 at the next level equals the current one. Requires s_min_cur >= s_min_next. */
flod_status flod_adjust_scale(float *s_opt, int64_t n, float s_min_cur, float s_min_next,
                              flod_stream stream);

/* Copies the workspace status bits to *out (waits for `stream`). */
flod_status flod_read_status(const void *ws, uint32_t *out, flod_stream stream);

/* Human-readable name of a status code (static string). */
const char *flod_status_string(flod_status s);

#ifdef __cplusplus
}
#endif
#endif /* FLOD_H */
