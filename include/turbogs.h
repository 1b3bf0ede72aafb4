/*
 * turbogs.h - C ABI of the GB300 sparse-sampled Gaussian-splatting path.
 *
 * The calls follow the per-iteration steps of TurboGS (ICML 2026, Alg. 1):
 * view selection (step 2: per-view error totals and the geometry-aware
 * draw), pixel sampling (step 3), sparse forward rendering (step 5), the
 * fused sparse loss with the error/age map update (steps 4, 6, 7), the sparse
 * backward (step 8), the hybrid update (steps 9, 10) and the error
 * back-projection statistics (step 11), plus the projection and tile binning
 * of the 3DGS rasterizer they run on (Sec. 3.1).
 *
 * Conventions (all entry points):
 *  - Every array argument is a DEVICE pointer owned by the caller, contiguous,
 *    row-major, aligned to 16 bytes.  float = IEEE binary32.  Nothing is
 *    allocated, freed or kept by the library; scratch is passed in as
 *    `workspace` of the size the matching *_workspace_size() call returns.
 *  - Calls are asynchronous on `stream` (a cudaStream_t; NULL = the legacy
 *    default stream) and never synchronise.  Counts produced on the device
 *    (n_active, n_isect) stay on the device; kernels size their grids from the
 *    host-side upper bounds passed in, so a sequence of calls can be captured
 *    in a CUDA graph.
 *  - Return value: TGS_OK, or an error code.  On TGS_ERR_INVALID_ARG nothing
 *    was launched and no memory was written.  On TGS_ERR_CUDA a launch failed;
 *    tgs_last_cuda_error() returns the CUDA error code.
 *  - Image geometry: pixel (x, y) covers [x, x+1) x [y, y+1) and is sampled at
 *    its centre (x + 0.5, y + 0.5).  Tiles are 16 x 16 pixels; tile id =
 *    ty * tiles_x + tx with tiles_x = ceil(width / 16).  A pixel is named
 *    inside its tile by its local index l = ly * 16 + lx (0..255).
 *  - Thread safety: calls keep no state and may be issued from any thread.
 */
#ifndef TURBOGS_H
#define TURBOGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* tgs_stream; /* = cudaStream_t */

typedef enum {
  TGS_OK = 0,
  TGS_ERR_INVALID_ARG = 1, /* bad pointer, size, alignment or option */
  TGS_ERR_CAPACITY = 2,    /* an output buffer is too small */
  TGS_ERR_CUDA = 3,        /* a CUDA launch or copy failed */
  TGS_ERR_TIMEOUT = 4,     /* a bounded device-side wait gave up */
  TGS_ERR_DEVICE = 5       /* no usable sm_103 device */
} tgs_status;

/* Pinhole camera.  viewmat: row-major 4x4 world-to-camera transform with
 * camera axes x right, y down, z forward.  fx, fy, cx, cy in pixels.  A
 * Gaussian is culled unless its camera-space depth z > znear. */
typedef struct {
  float viewmat[16];
  float fx, fy, cx, cy;
  int32_t width, height;
  float znear;
} tgs_camera;

/* N Gaussians (Sec. 3.1: centre, covariance via scale and rotation,
 * opacity, colour coefficients).
 *   means [N,3], log_scales [N,3] (scale = exp), quats [N,4] (w, x, y, z; the
 *   rotation of q/|q|), opacity_logits [N] (opacity = sigmoid), sh [N,16,3]
 *   (real spherical harmonics of degree <= 3, coefficient-major, RGB inner).
 * Only the first (sh_degree+1)^2 coefficients are used.
 * geo_stride: 0 for four packed arrays (3, 3, 4 and 1 floats per Gaussian);
 * otherwise the distance in floats between consecutive Gaussians of all four
 * geometric fields, which then lie in one array of rows (a multiple of 4, at
 * least 12; e.g. 16: means at row + 0, log_scales at + 3, opacity_logits at
 * + 6, quats at + 8, one 64-byte row per Gaussian, so that an update of
 * scattered Gaussians reads and writes whole rows).  quats stays 16-byte
 * aligned.  sh is always [N,16,3]. */
typedef struct {
  const float* means;
  const float* log_scales;
  const float* quats;
  const float* opacity_logits;
  const float* sh;
  int64_t n;
  int32_t sh_degree;
  int32_t geo_stride;
} tgs_gaussians;

/* Mutable arrays with the layout of tgs_gaussians (parameters, gradients,
 * first and second moments), geo_stride as there. */
typedef struct {
  float* means;
  float* log_scales;
  float* quats;
  float* opacity_logits;
  float* sh;
  int32_t geo_stride;
} tgs_param_ptrs;

/* Screen-space splats, the output of the projection:
 *   xy [N,2] centre in pixel coordinates; conic_opac [N,4] = (a, b, c, o) with
 *   [[a, b], [b, c]] the inverse 2D covariance and o the opacity; rgb [N,3];
 *   depth [N] camera-space z; radius [N] in pixels, 0 when culled. */
typedef struct {
  float* xy;
  float* conic_opac;
  float* rgb;
  float* depth;
  int32_t* radius;
} tgs_projected;

/* Split of the sampled set, in units of 1/1000 (TurboGS Table 6: hard 0.4,
 * stable 0.3, remainder mixed). */
typedef struct {
  int32_t tile_hard_pm, tile_stable_pm;
  int32_t pix_hard_pm, pix_stable_pm;
} tgs_sampling;

/* Loss constants (Sec. 3.7, App. A): Charbonnier epsilon, NCC epsilon, EMA
 * ratio beta (Table 6: 0.4).  view_weight scales this view's loss and
 * dL_drgb: 1 for one view, 1/K for the mean over K views of one step (the
 * expectation over views in Eq. 11). */
typedef struct {
  float eps_charbonnier, eps_ncc, beta, view_weight;
} tgs_loss_params;

/* Hybrid solver (Sec. 3.9, App. A).  lr: means, log_scales, quats, opacity,
 * SH DC, SH rest.  mode: 0 Adam on all parameters; 1 LM blocks with the
 * diagonal of J^T J; 2 LM blocks with the full J^T J solved by Cholesky. */
typedef struct {
  float lr[6];
  float beta1, beta2, eps_adam, eps_lm;
  int32_t mode;
} tgs_opt;

/* Library version string and CUDA error of the last failed call (per thread). */
const char* tgs_version(void);
int32_t tgs_last_cuda_error(void);
const char* tgs_status_string(int32_t status);

/* Checks that the current device can run the library's sm_103a code. */
tgs_status tgs_device_check(void);

/* Number of kernel nodes in a captured CUDA graph (a cudaGraph_t passed as
 * void*), or -1 on error; for counting the kernels one replay launches. */
int64_t tgs_graph_count_kernels(void* graph);

/*
 * select_tiles - tile selection and tile-wise error-guided pixel sampling
 * (Sec. 3.5, Eqs. 7-8; Alg. 1 step 3).
 *
 * Chooses n_sel = min(n_select, T) of the T tiles of one view, then in each
 * chosen tile N_pix = min(n_pix, valid pixels of the tile) pixels.  Each level
 * takes round(r_hard n) items by the error-proportional draw without
 * replacement (pixel weight = fp16 E * 2^24, tile weight = sum over its
 * pixels), then round(r_stable n) of the rest with the largest age (a tile's
 * age is its smallest pixel age), then the remainder uniformly.  The draws use
 * the counter-based SplitMix64 hash of (seed, iter, view, stream, tile, item);
 * the weighted draw is the Efraimidis-Spirakis order of E_i / w_i with E_i an
 * exponential variate in 32-bit fixed point.  Ties go to the lower index.
 * Results are bit-identical on every run for the same inputs.
 *
 *   err_map [H,W]  fp16 error map E_v (bit patterns); negative, NaN and
 *                  infinite values count as 0
 *   age_map [H,W]  uint16 age map A_v
 *   n_pix          1..256
 *   iter_dev       nullable device uint64: when given, the iteration number is
 *                  read from it at run time instead of `iter` (for replays of
 *                  a captured graph)
 *   workspace      tgs_select_tiles_workspace_size(width, height) bytes
 * Outputs: active_tiles [n_sel] (ascending tile ids), n_active [1],
 * tile_rank [T] (index into active_tiles, -1 when not chosen),
 * pix_off [n_sel+1] (prefix offsets), pix_idx [n_sel * n_pix] (local pixel
 * indices, ascending within each tile).
 */
size_t tgs_select_tiles_workspace_size(int32_t width, int32_t height);
tgs_status tgs_select_tiles(const uint16_t* err_map, const uint16_t* age_map, int32_t width, int32_t height,
                            int32_t n_select, int32_t n_pix, const tgs_sampling* cfg, uint64_t seed,
                            uint64_t iter, const uint64_t* iter_dev, uint32_t view, void* workspace,
                            size_t workspace_bytes,
                            int32_t* active_tiles, int32_t* n_active, int32_t* tile_rank, int32_t* pix_off,
                            uint8_t* pix_idx, tgs_stream stream);

/*
 * select_tiles_noalloc - the same selection as tgs_select_tiles, for callers
 * that cannot allocate device memory (the paper has no counterpart: this is a
 * deployment variant).  Some hosts own all device memory and forbid any other
 * allocation (a fixed pool handed out by a framework, an embedded runtime),
 * and on latency-critical paths an allocation may block or synchronise.  This
 * entry point takes no workspace: its scratch is one device array of
 * TGS_SELECT_NOALLOC_SCRATCH_BYTES compiled into the library, which every GPU
 * that loads the library holds until the process exits.  Nothing is
 * allocated or freed by the call.
 *   - Views of more than TGS_SELECT_NOALLOC_MAX_TILES tiles are rejected with
 *     TGS_ERR_CAPACITY before anything is launched.
 *   - The first call on a device looks up the array's device address (with
 *     that device current) and caches it; make that first call before any
 *     stream capture.  The cached address belongs to the device's current
 *     context: after cudaDeviceReset (or any teardown of the primary context)
 *     the library's module is loaded again and the array may move, so a
 *     process that resets a device must not call this entry point on it
 *     again.
 *   - Devices with an ordinal of TGS_SELECT_NOALLOC_MAX_DEVICES or more get
 *     TGS_ERR_CAPACITY (the address cache has that many entries).
 *   - All calls on a device share the one array, and it keeps the last
 *     call's contents (the call clears what must start at zero itself).  Calls
 *     that can overlap on the GPU (different streams, or different host
 *     threads without ordering) race on it: order them on one stream.
 * Arguments and outputs are those of tgs_select_tiles without the workspace.
 */
#define TGS_SELECT_NOALLOC_MAX_TILES 16384
#define TGS_SELECT_NOALLOC_SCRATCH_BYTES (768u * 1024u)
#define TGS_SELECT_NOALLOC_MAX_DEVICES 64
tgs_status tgs_select_tiles_noalloc(const uint16_t* err_map, const uint16_t* age_map, int32_t width,
                                    int32_t height, int32_t n_select, int32_t n_pix, const tgs_sampling* cfg,
                                    uint64_t seed, uint64_t iter, const uint64_t* iter_dev, uint32_t view,
                                    int32_t* active_tiles, int32_t* n_active, int32_t* tile_rank, int32_t* pix_off,
                                    uint8_t* pix_idx, tgs_stream stream);

/*
 * view_error_sums - the per-view error totals behind the anchor choice of
 * geometry-aware view sampling (Sec. 3.4, Eq. 5: the mean of E_v over the
 * image domain, which is this sum divided by W H).
 *
 *   err_maps   device fp16 error maps (bit patterns), view v at
 *              err_maps + v * view_stride, each [H,W] row-major; negative,
 *              NaN and infinite values count as 0 (as in select_tiles)
 *   sums [V]   device out: sum over the view's pixels of E * 2^24, exact in
 *              integers (every fp16 value is an integer multiple of 2^-24)
 * Requires 1 <= n_views, width, height; W H <= 2^23 (so a sum stays below
 * 2^63); view_stride >= W H.  The 16-byte path is taken when err_maps and
 * view_stride * 2 are multiples of 16 and W H of 8.  sums is overwritten.
 * Results are independent of the launch order (integer addition).
 */
#define TGS_VIEW_MAX_PIXELS (1 << 23)
tgs_status tgs_view_error_sums(const uint16_t* err_maps, int32_t n_views, int64_t view_stride, int32_t width,
                               int32_t height, uint64_t* sums, tgs_stream stream);

/*
 * sample_views - geometry-aware view sampling (Sec. 3.4, Eqs. 5-6; Alg. 1
 * step 2): K views for one iteration, drawn without replacement from a view
 * stack.
 *   1. If fewer than K views are on the stack, every view is put back on it
 *      (the refill; the draw below is by weight, so the reshuffle the paper
 *      pairs with it has no effect and is not a separate step).
 *   2. The anchor v* is the stack view with the largest error sum (Eq. 5;
 *      equal sums go to the lower index).
 *   3. The other K - 1 are drawn from the remaining stack views, one after
 *      another, each with probability proportional to
 *        pi(u) = exp(-lambda_d |c_u - c_v*| - lambda_theta (1 - <d_u, d_v*>))
 *      (Eq. 6), c_u the camera centre -R^T t and d_u its unit forward axis
 *      (the third row of R, normalised) from cams[u].viewmat.  The draws are
 *      the K - 1 smallest Efraimidis-Spirakis keys
 *        log2(-log2 U_u) + log2(e) (lambda_d |c_u - c_v*| + lambda_theta (1 - <d_u, d_v*>))
 *      with -log2 U_u from the SplitMix64 hash of (seed, iter, stream 5,
 *      item u) in 32-bit fixed point and its log2 by the same digit
 *      recurrence; everything else in IEEE double without fused operations,
 *      so a run gives the same views on every machine.  Equal keys go to the
 *      lower index.
 *   4. The K views leave the stack.
 *
 *   err_sums [V]  device, from tgs_view_error_sums (or any non-negative totals)
 *   cams [V]      device camera array
 *   stack [V]     device uint8 in/out: 1 while the view is on the stack
 *                 (start with all ones)
 *   views [K]     device out: views[0] = v*, then the K - 1 draws ascending
 * Requires 1 <= K <= V <= TGS_VIEW_SAMPLE_MAX_VIEWS and finite, non-negative
 * lambda_d, lambda_theta.
 */
#define TGS_VIEW_SAMPLE_MAX_VIEWS 8192
tgs_status tgs_sample_views(const uint64_t* err_sums, const tgs_camera* cams, int32_t n_views, int32_t k,
                            double lambda_d, double lambda_theta, uint64_t seed, uint64_t iter, uint8_t* stack,
                            int32_t* views, tgs_stream stream);

/*
 * project_gaussians - EWA projection and SH colour of the 3DGS model the
 * method rasterizes (Sec. 3.1).
 *
 * Sigma = R diag(exp(2 log_scale)) R^T; camera-space centre t = W mu + T; culled
 * unless t.z > znear; Sigma2 = J W Sigma W^T J^T + 0.3 I with the perspective
 * Jacobian J (x/z, y/z clamped to 1.3 times the half field of view); culled
 * unless det Sigma2 > 0; radius = ceil(3 sqrt(lambda_max)),
 * lambda_max = m + sqrt(max(0.1, m^2 - det)), m = trace/2; culled when its
 * 16-pixel tile rectangle (tiles k with 16k <= c + r and 16k + 16 > c - r, decided
 * in single precision) is empty or, when tile_rank is given, holds no tile with
 * tile_rank >= 0.  rgb = max(0, sum_k sh_k Y_k(d) + 0.5) with d the unit
 * direction from the camera centre; opacity = sigmoid(logit).
 * Culled Gaussians get radius 0 and zeros elsewhere.
 */
tgs_status tgs_project_gaussians(const tgs_gaussians* g, const tgs_camera* cam, const int32_t* tile_rank,
                                 tgs_projected* out, tgs_stream stream);

/*
 * bin_tiles - per-tile Gaussian lists sorted by depth (Sec. 3.1, the ordered
 * sets K(p)): every (active tile, Gaussian) pair whose tile rectangle covers
 * the tile, ordered by (tile, depth, Gaussian id): a counting sort on the
 * active-tile rank (shared-memory histograms per chunk of Gaussians) and a
 * sort within each tile.  When capacity exceeds 2048 pairs per tile of the
 * view (long lists), the Gaussians are first radix-sorted by depth so that
 * only short segments of each list need sorting; the result is the same.
 *
 *   proj        xy, depth, radius of the projection (radius 0 = skip)
 *   tile_rank   [T] active-tile index or -1 (NULL: every tile active, rank = id)
 *   n_active_max  number of ranks (T when tile_rank is NULL)
 *   capacity    length of vals / keys
 * Outputs: vals [capacity] Gaussian ids in order; keys [capacity] (nullable)
 * = tile id << 32 | float bits of depth; tile_ranges [n_active_max, 2]
 * half-open [start, end) per rank; n_isect [1] = number of pairs.  If
 * n_isect > capacity only the first `capacity` pairs in emission order are
 * kept, the sort and ranges are then invalid: the caller checks n_isect and
 * retries with more capacity.
 */
size_t tgs_bin_tiles_workspace_size(int64_t n, int64_t capacity, int32_t n_active_max);
tgs_status tgs_bin_tiles(const tgs_projected* proj, int64_t n, const tgs_camera* cam, const int32_t* tile_rank,
                         int32_t n_active_max, void* workspace, size_t workspace_bytes, int64_t capacity,
                         int32_t* vals, uint64_t* keys, int32_t* tile_ranges, int64_t* n_isect, tgs_stream stream);

/*
 * Checkpoints of the sampled forward (not in the paper: they let the
 * backward of Sec. 3.6 replay one tile's list in several independent pieces,
 * so a sparse step has enough parallel work).  Slot c of sampled pixel s
 * holds float4 (T, C_r, C_g, C_b): the transmittance and accumulated colour
 * in front of tile-list position 32 (c + 1), at data[(c * stride + s) * 4],
 * written by every pixel whose walk reaches that position (the others' slots
 * are never read).  data: device, 16-byte aligned,
 * tgs_checkpoint_bytes(n_active_max, n_pix_max, n_slots) bytes;
 * stride >= n_active_max * n_pix_max.  rgb: the forward's rgb output (the
 * backward reads it).  Pass the same struct to render_sampled and
 * backward_sampled with the same n_pix_max, or NULL to both.
 */
typedef struct {
  float* data;
  int32_t n_slots;
  int64_t stride;
  const float* rgb;
  int32_t* tile_last;  /* nullable [n_active_max]: per active rank, the longest
                          blended run of its pixels (written by the forward, lets
                          the backward skip empty pieces without reading n_last) */
} tgs_checkpoints;

size_t tgs_checkpoint_bytes(int32_t n_active_max, int32_t n_pix_max, int32_t n_slots);

/*
 * set_forward_split - a tuning knob of render_sampled with checkpoints (not in
 * the paper).  With checkpoints and few active tiles, the forward walks each
 * tile's list in NW runs of 32 positions at once (NW groups of one thread per
 * sampled pixel, each run from a local transmittance of 1) and composes the
 * runs' results in list order, (T, C) -> (T T_run, C + T C_run); the run in
 * which the composed transmittance falls below the stopping value is walked
 * again from its entry state to find the exact stop.  The result equals the
 * sequential walk up to the rounding of the composition.  groups = 3 takes
 * the sequential walk with every warp on its own (each stages its own splat
 * batches and stops when its own pixels have saturated; the same bits as
 * the sequential walk), several tiles per block when tiles have few sampled
 * pixels.  groups = 0 (the default) leaves the choice to the library (the
 * walk with two threads per pixel for sparse launches of tiles with at most
 * 32 sampled pixels, else the block's walk); 1 is the block's sequential walk; 2 or 4
 * the split walk; 5 the walk with two threads per pixel (each walks one half
 * of every 32-position run at once, the second from a local transmittance of
 * 1; the halves compose as above, and the second half walks again from the
 * composed state where the stop may lie in it, so that the stops and n_last
 * are the sequential walk's).
 * Process-wide; returns TGS_ERR_INVALID_ARG for other values.
 */
tgs_status tgs_set_forward_split(int32_t groups);

/*
 * render_sampled - sparse forward rasterization (Sec. 3.6, Eq. 1; Alg. 1
 * step 5): for every sampled pixel of every active tile, front-to-back
 * compositing over the tile's list: alpha = min(0.99, o exp(power)),
 * power = -(a dx^2 + c dy^2)/2 - b dx dy at the pixel centre; splats with
 * power > 0 or alpha < 1/255 are skipped; the walk stops before the splat
 * that would take the transmittance below 1e-4.
 *
 *   active_tiles / n_active / pix_off / pix_idx   as from select_tiles
 *   n_active_max, n_pix_max   host-side bounds (grid and block sizes)
 *   bg [3]  host array, background colour
 * Outputs per sampled pixel s (tile order): rgb [P,3] = sum T alpha c + T bg,
 * T_final [P], n_last [P] = 1 + position in the tile list of the last splat
 * blended (0 if none).
 */
tgs_status tgs_render_sampled(const tgs_projected* proj, const int32_t* tile_ranges, const int32_t* vals,
                              const int32_t* active_tiles, const int32_t* n_active, int32_t n_active_max,
                              const int32_t* pix_off, const uint8_t* pix_idx, int32_t n_pix_max,
                              const tgs_camera* cam, const float* bg, float* rgb, float* T_final,
                              int32_t* n_last, const tgs_checkpoints* ckpt, tgs_stream stream);

/*
 * loss_sparse_ncc - fused sparse supervision (Sec. 3.7, Eqs. 9-11; App. A;
 * Alg. 1 steps 4, 6, 7), one thread block per active tile:
 *   l1(p) = sum_c sqrt((x - y)^2 + eps_c^2);
 *   NCC_c = cov / sqrt(var_x var_y + eps_n) over the tile's sampled pixels;
 *   lambda_tau = clip(mean_p |dl1/dx|_1 / (mean_p |n dNCC/dx|_1 + 1e-8), 0, 1);
 *   L = (1/P) sum_p l1(p) + (1/A) sum_tau lambda_tau (1 - mean_c NCC_c),
 *   lambda held constant in the gradient.
 * Writes dL_drgb [P,3], lambda_tile [n_active], err_pix [P] = sum_c |x - y|
 * (Eq. 2) and *loss (device double, overwritten).  When given, updates the
 * error map E <- fp16((1 - beta) E + beta e) at sampled pixels (Eq. 3) and the
 * age map A <- A + 1 (saturating at 65535) at every pixel, 0 at sampled
 * pixels (Eq. 4).  target [H,W,3] float.
 */
tgs_status tgs_loss_sparse_ncc(const float* rgb, const float* target, int32_t width, int32_t height,
                               const int32_t* active_tiles, const int32_t* n_active, int32_t n_active_max,
                               const int32_t* pix_off, const uint8_t* pix_idx, int32_t n_pix_max,
                               const tgs_loss_params* params, uint16_t* err_map, uint16_t* age_map,
                               float* dL_drgb, float* lambda_tile, float* err_pix, double* loss,
                               tgs_stream stream);

/*
 * loss_sparse_ssim - the same fused loss with the structure term of Table 4's
 * S-SSIM variant in place of the sparse NCC (the paper names the variant
 * only; this is its reading): per active tile and colour channel, SSIM
 * (Wang et al. 2004, C1 = 0.01^2, C2 = 0.03^2) from population moments over
 * the tile's sampled pixels, S-SSIM_tau = 1 - mean_c SSIM_c, weighted by the
 * same clipped gradient ratio lambda_tau (with n dSSIM/dx in place of the NCC
 * derivative).  params->eps_ncc is not used.  Everything else (Charbonnier L1,
 * e, the error and age map updates, arguments, outputs, errors) is as
 * loss_sparse_ncc.
 */
tgs_status tgs_loss_sparse_ssim(const float* rgb, const float* target, int32_t width, int32_t height,
                                const int32_t* active_tiles, const int32_t* n_active, int32_t n_active_max,
                                const int32_t* pix_off, const uint8_t* pix_idx, int32_t n_pix_max,
                                const tgs_loss_params* params, uint16_t* err_map, uint16_t* age_map,
                                float* dL_drgb, float* lambda_tile, float* err_pix, double* loss,
                                tgs_stream stream);

/*
 * error_stats_sampled - error back-projection statistics (Sec. 3.8, Eq. 12;
 * Alg. 1 step 11), a pass of its own after the loss.  For
 * every sampled pixel p and every splat k it blended (list positions below
 * n_last, alpha as render_sampled computes it), with compositing weight
 * w = T_k alpha_k and D = sqrt(a dx^2 + 2 b dx dy + c dy^2) the conic
 * Mahalanobis distance of the pixel centre from the splat, adds
 * (e(p) w, w, D w, 0) to stats [n_gaussians, 4] (device float, 16-byte
 * aligned; zeroed first unless accumulate = 1, which sums over the views of
 * an iteration).  err_pix [P]: the per-pixel error e(p) (as loss_sparse_ncc
 * writes it); n_last [P]: as render_sampled writes it.  Other arguments as in
 * render_sampled.  The normalised statistics E / (W + eps), D / (W + eps)
 * are left to the caller.
 */
tgs_status tgs_error_stats_sampled(const tgs_projected* proj, const int32_t* tile_ranges, const int32_t* vals,
                                   const int32_t* active_tiles, const int32_t* n_active, int32_t n_active_max,
                                   const int32_t* pix_off, const uint8_t* pix_idx, int32_t n_pix_max,
                                   const tgs_camera* cam, const int32_t* n_last, const float* err_pix,
                                   float* stats, int64_t n_gaussians, int32_t accumulate, tgs_stream stream);

/*
 * backward_sampled - sparse backward (Sec. 3.6; Alg. 1 step 8).  Replays each
 * sampled pixel's compositing in reverse from T_final and n_last, recovering
 * T_k = T_{k+1} / (1 - alpha_k), and accumulates the adjoints of the screen-
 * space splats (dL/dc_k = T_k alpha_k g, dL/dalpha_k = T_k (c_k - S_{k+1}) . g
 * with S the colour seen behind), reduced across each warp with shuffles
 * before one vector atomic per warp and splat, into grad2d [N,12]
 * (caller scratch, zeroed here): (dx, dy, da, db | dc, dopacity, dr, dg |
 * db(blue), 0, 0, 0).  Then the projection adjoint maps it to gradients of
 * the parameters (grads, layout of tgs_gaussians) and touched [N] = 1 where
 * grad2d is not all zero.  write_untouched = 0 leaves grads of untouched
 * Gaussians unwritten; 1 writes zeros there.  With checkpoints (ckpt, as
 * given to render_sampled) each tile's list is replayed in independent pieces
 * of 32 positions, one warp each over all of the tile's sampled pixels, every
 * piece starting from the forward's checkpoint at its back edge
 * (S = (rgb - C) / T there), or from (T_final, bg) for the piece holding the
 * pixel's last splat; the positions past the last slot form one more piece.
 * Same result up to rounding; more parallel work for sparse steps.
 */
tgs_status tgs_backward_sampled(const tgs_gaussians* g, const tgs_camera* cam, const tgs_projected* proj,
                                const int32_t* tile_ranges, const int32_t* vals, const int32_t* active_tiles,
                                const int32_t* n_active, int32_t n_active_max, const int32_t* pix_off,
                                const uint8_t* pix_idx, int32_t n_pix_max, const float* bg, const float* T_final,
                                const int32_t* n_last, const float* dL_drgb, float* grad2d,
                                const tgs_param_ptrs* grads, uint8_t* touched, int32_t write_untouched,
                                const tgs_checkpoints* ckpt, tgs_stream stream);

/*
 * render_backward_sampled - the first half of backward_sampled alone: zeroes
 * grad2d [n_gaussians, 12] and accumulates the compositing adjoint into it
 * (arguments as in backward_sampled).
 */
tgs_status tgs_render_backward_sampled(const tgs_projected* proj, const int32_t* tile_ranges, const int32_t* vals,
                                       const int32_t* active_tiles, const int32_t* n_active, int32_t n_active_max,
                                       const int32_t* pix_off, const uint8_t* pix_idx, int32_t n_pix_max,
                                       const tgs_camera* cam, const float* bg, const float* T_final,
                                       const int32_t* n_last, const float* dL_drgb, float* grad2d,
                                       int64_t n_gaussians, const tgs_checkpoints* ckpt, tgs_stream stream);

/*
 * render_backward_sampled_stats - render_backward_sampled, and in the same
 * replay the error back-projection statistics of Sec. 3.8 (Eq. 12; Alg. 1
 * step 11) over the same sampled pixels: for every splat a pixel blends with
 * compositing weight w = T alpha, stats[i] += (e w, w, D w, 0), with e the
 * pixel's error err_pix [P] (from loss_sparse_ncc) and D the conic
 * Mahalanobis distance of the pixel centre from the splat.  The weights are
 * the ones the backward recovers (T by division from the end of the walk),
 * equal to the forward's up to rounding.  stats: device [N,4] float, 16-byte
 * aligned, zeroed first unless accumulate_stats = 1 (so the views of a step
 * and several steps can add up).  With checkpoints the sums ride on the
 * warp-per-piece replay (one more 4-value warp reduction and one vector
 * atomic per warp and splat); without, error_stats_sampled runs after the
 * whole-tile backward.  Other arguments and results as
 * render_backward_sampled.
 */
tgs_status tgs_render_backward_sampled_stats(const tgs_projected* proj, const int32_t* tile_ranges,
                                             const int32_t* vals, const int32_t* active_tiles,
                                             const int32_t* n_active, int32_t n_active_max, const int32_t* pix_off,
                                             const uint8_t* pix_idx, int32_t n_pix_max, const tgs_camera* cam,
                                             const float* bg, const float* T_final, const int32_t* n_last,
                                             const float* dL_drgb, float* grad2d, int64_t n_gaussians,
                                             const tgs_checkpoints* ckpt, const float* err_pix, float* stats,
                                             int32_t accumulate_stats, tgs_stream stream);

/*
 * accumulate_screen_grad - the screen-space gradient statistic that selects
 * densification candidates (Alg. 1 step 11 takes the screen-space gradients;
 * Table 6's tau_grad): for every Gaussian whose grad2d row [N,12] (one view,
 * as render_backward_sampled writes it) is not all zero,
 * accum[i] += (|(dL/dx, dL/dy)|, 1), in single precision (sqrt of the sum of
 * squares, IEEE-rounded).  grad2d: device, 16-byte aligned; accum: device
 * [N,2] float, 8-byte aligned, added to (zero it after a density step).
 */
tgs_status tgs_accumulate_screen_grad(const float* grad2d, int64_t n, float* accum, tgs_stream stream);

/*
 * density_control - one step of error-driven densification and pruning
 * (Sec. 3.8, Eq. 13; Alg. 1 step 11; Table 6).  The paper fixes the
 * difficulty score and says that percentile thresholds of it drive the
 * density control; this is the procedure as read here, every decision an
 * IEEE single-precision operation in this order:
 *   e_i = E_i / (W_i + eps), d_i = D_i / (W_i + eps), s_i = e_i + lambda_eff d_i
 *   (stats rows (E, W, D, -) of Eq. 12; lambda_eff = lambda_base (1 - rho)
 *   computed by the caller); g_i = accum_i.x / max(1, accum_i.y);
 *   pruned: opacity logit < opacity_logit_prune;
 *   candidates: not pruned, W_i > 0 and g_i >= tau_grad;
 *   densified: the floor(n_candidates topk_permille / 1000) candidates with
 *   the largest s_i (equal scores: the lower index first);
 *   a densified Gaussian is cloned (an identical copy follows it) when its
 *   largest log-scale is at most log_scale_split, else split into two
 *   children at mu +- sigma_k (R e_k) (k: the axis of the largest scale, the
 *   lower axis on ties; R the rotation of the normalised quaternion) with
 *   every log-scale lowered by ln 1.6;
 *   final_prune = 1 (the final pruning of Table 6): nothing is densified and
 *   every Gaussian outside the floor(N final_permille / 1000) with the
 *   largest W_i (ties: lower index) is pruned as well.
 * Inputs: the parameters (g, n = g->n < 2^31), moments m_in, v_in (layout of
 * tgs_gaussians), stats [N,4] (16-byte aligned), accum [N,2] (8-byte
 * aligned).  Outputs, in input order (each surviving Gaussian in place, a
 * clone's copy or a split's second child right after it): parameters and
 * moments g_out, m_out, v_out with room for `capacity` Gaussians (the copy
 * and both children start from zero moments; the rest keep theirs),
 * n_out (device) = the output count, which may exceed capacity (then rows
 * past it are not written: retry with more), src_out (device, nullable)
 * [capacity] = the input index of every output row.  Outputs must not alias
 * inputs.  workspace: density_control_workspace_size(N) bytes.
 */
typedef struct {
  float lambda_eff;          /* lambda_base (1 - rho) of Eq. 13 */
  float eps;                 /* Eq. 13's epsilon */
  float tau_grad;            /* Table 6: gradient threshold for densification */
  float log_scale_split;     /* log of the clone/split size (Table 6's percent dense x scene extent) */
  float opacity_logit_prune; /* logit of the pruning opacity */
  int32_t topk_permille;     /* Table 6: fraction for top-k densification, x 1000 */
  int32_t final_prune;       /* 1: the final pruning step, 0: densify and prune */
  int32_t final_permille;    /* Table 6: fraction retained by the final pruning, x 1000 */
} tgs_density_params;

size_t tgs_density_control_workspace_size(int64_t n);
tgs_status tgs_density_control(const tgs_gaussians* g, const tgs_param_ptrs* m_in, const tgs_param_ptrs* v_in,
                               const float* stats, const float* accum, const tgs_density_params* cfg,
                               const tgs_param_ptrs* g_out, const tgs_param_ptrs* m_out,
                               const tgs_param_ptrs* v_out, int64_t capacity, int64_t* n_out, int64_t* src_out,
                               void* workspace, size_t workspace_bytes, tgs_stream stream);

/*
 * project_backward - the projection adjoint alone (the second half of
 * backward_sampled, Alg. 1 step 8): grad2d [N,12] of one view -> parameter
 * gradients.  accumulate = 0 overwrites grads and touched as backward_sampled
 * does.  accumulate = 1 sums views of one step: touched (required) must be
 * zeroed before the first view; a Gaussian this view touches gets its
 * gradient written when touched[i] is still 0 and added otherwise, and
 * touched[i] becomes 1 (untouched gradients are left alone: the update reads
 * only touched Gaussians).  view_row (nullable, 8-byte aligned) receives this
 * view's own [N,14] gradient row in the hybrid_step layout (means, log-scales,
 * quaternion, DC r g b, opacity logit; zeros where untouched), i.e. one
 * K-slice of its view_rows.
 */
tgs_status tgs_project_backward(const tgs_gaussians* g, const tgs_camera* cam, const tgs_projected* proj,
                                const float* grad2d, const tgs_param_ptrs* grads, uint8_t* touched,
                                int32_t write_untouched, int32_t accumulate, float* view_row, tgs_stream stream);

/*
 * project_backward_multi - the projection adjoint of K views of one step
 * (1 <= K <= 16) in one pass: each Gaussian's parameters are read once, the
 * adjoints of the views whose grad2d row is non-zero are summed in registers
 * and the gradients are written once (so the result is the sum over views of
 * project_backward).  Per view v: cams[v], radius[v] (that view's projection
 * output), grad2d[v] [N,12] (16-byte aligned) and, when view_rows is given
 * and view_rows[v] is not NULL, view_rows[v] [N,14] as in project_backward.
 * The pointer arrays are host arrays of device pointers.  touched[i] (may be
 * NULL) = 1 when any view touched Gaussian i; untouched gradients are zeroed
 * only with write_untouched.  workspace: 16-byte aligned device scratch of
 * tgs_project_backward_multi_workspace_size(N) bytes (the list of touched
 * Gaussians, processed in a second pass).
 */
size_t tgs_project_backward_multi_workspace_size(int64_t n);
tgs_status tgs_project_backward_multi(const tgs_gaussians* g, int32_t n_views, const tgs_camera* cams,
                                      const int32_t* const* radius, const float* const* grad2d,
                                      const tgs_param_ptrs* grads, uint8_t* touched, int32_t write_untouched,
                                      float* const* view_rows, void* workspace, size_t workspace_bytes,
                                      tgs_stream stream);

/*
 * project_backward_update - project_backward_multi followed by hybrid_step in
 * one pass (modes 0 and 1 of tgs_opt, whose update of a Gaussian needs only
 * its own summed gradient): for each Gaussian that a view touched, the sum
 * of the views' projection adjoints is formed in registers and shared memory
 * and the Gaussian's parameters (params, in place), m and v are updated at
 * once; no gradient is written.  touched as in project_backward_multi;
 * workspace: tgs_project_backward_multi_workspace_size(n) bytes, 16-byte
 * aligned.  Mode 2 (per-view Jacobian rows, Cholesky) is rejected: use
 * project_backward_multi with view_rows and hybrid_step.
 */
tgs_status tgs_project_backward_update(const tgs_param_ptrs* params, int64_t n, int32_t sh_degree, int32_t n_views,
                                       const tgs_camera* cams, const int32_t* const* radius,
                                       const float* const* grad2d, const tgs_param_ptrs* m, const tgs_param_ptrs* v,
                                       uint8_t* touched, const tgs_opt* opt, int32_t step, const int32_t* step_dev,
                                       void* workspace, size_t workspace_bytes, tgs_stream stream);

/*
 * Several views in one launch (not in the paper: a batching of
 * render_sampled / the compositing adjoint over the views of one iteration,
 * Alg. 1 steps 5 and 8).  Persistent thread blocks (grid_ctas of them) take
 * (view, active tile) items from an atomic counter (counter: one device
 * int32, reset by the call) until none are left; each item is rendered
 * exactly as render_sampled / backward_sampled render it.  Up to 16 views.
 * Per view: the fields of render_sampled; the backward also reads dL_drgb
 * and writes grad2d [n_gaussians, 12] (zeroed by the call).  With checkpoints
 * (ckpt.data, rgb = the view's rgb output) the forward stores them and the
 * backward replays every tile in pieces as backward_sampled does, each warp
 * of the persistent blocks taking its own (view, tile, piece) items.
 */
typedef struct {
  tgs_projected proj;
  const int32_t* tile_ranges;
  const int32_t* vals;
  const int32_t* active_tiles;
  const int32_t* n_active;
  int32_t n_active_max;
  const int32_t* pix_off;
  const uint8_t* pix_idx;
  int32_t n_pix_max;
  tgs_camera cam;
  float bg[3];
  float* rgb;
  float* T_final;
  int32_t* n_last;
  const float* dL_drgb;
  float* grad2d;
  int64_t n_gaussians;
  tgs_checkpoints ckpt;  /* n_slots = 0: none; else the same n_slots in every view */
} tgs_view_batch;

/* Advances the device-side iteration counters of a captured step by one
 * (iter_dev as read by select_tiles, step_dev as read by hybrid_step; either
 * may be NULL).  Not in the paper: the counters let one captured step be
 * replayed. */
tgs_status tgs_advance_counters(int64_t* iter_dev, int32_t* step_dev, tgs_stream stream);

/* Thread blocks of the batched kernels that fit on the current device at
 * once (SMs x resident blocks per SM) for n_pix_max pixels per tile: the
 * largest useful grid_ctas.  backward: 0 the forward, 1 the backward without
 * checkpoints (whole tiles), 2 the backward in pieces (with checkpoints). */
tgs_status tgs_render_batched_resident(int32_t n_pix_max, int32_t backward, int32_t* ctas);
tgs_status tgs_render_sampled_batched(const tgs_view_batch* views, int32_t n_views, int32_t grid_ctas,
                                      int32_t* counter, tgs_stream stream);
tgs_status tgs_render_backward_batched(const tgs_view_batch* views, int32_t n_views, int32_t grid_ctas,
                                       int32_t* counter, tgs_stream stream);
/* The batched backward with Eq. 12's statistics over the sampled pixels of
 * every view of the batch (Sec. 3.8: the sums run over the views and pixels
 * of the iteration), as render_backward_sampled_stats does for one view.
 * err_pix: host array [n_views] of device pointers to each view's per-pixel
 * errors; stats: device [n_gaussians,4] float shared by the views, 16-byte
 * aligned, zeroed first unless accumulate_stats = 1. */
tgs_status tgs_render_backward_batched_stats(const tgs_view_batch* views, int32_t n_views, int32_t grid_ctas,
                                             int32_t* counter, const float* const* err_pix, float* stats,
                                             int64_t n_gaussians, int32_t accumulate_stats, tgs_stream stream);

/*
 * hybrid_step - moment-damped LM / Adam update (Sec. 3.9, Eq. 14; App. A;
 * Alg. 1 steps 9, 10) of the Gaussians with touched[i] != 0.
 * m <- b1 m + (1 - b1) g, v <- b2 v + (1 - b2) g^2 on every parameter; the
 * geometry block (means, log_scales, quats: 10) and the appearance block (SH
 * DC rgb, opacity: 4) each solve (J^T J + diag(sqrt(v) + eps_lm)) D = -m
 * (mode 1: diagonal of J^T J; mode 2: full, Cholesky) and add lr * D; J is
 * view_rows [k_rows, N, 14] (geometry 10, then DC r g b and opacity), or the
 * gradient itself when view_rows is NULL.  The 45 higher SH coefficients (and
 * everything in mode 0) take the bias-corrected Adam step
 * -lr m_hat / (sqrt(v_hat) + eps_adam) at step `step` (>= 1), or, when
 * step_dev (device int32) is given, at the step read from it at run time.
 * touched may be NULL (every Gaussian updated).  The touched Gaussians are
 * first compacted into a list in `workspace`
 * (tgs_hybrid_step_workspace_size(n) bytes), so the update kernels run dense.
 */
size_t tgs_hybrid_step_workspace_size(int64_t n);
tgs_status tgs_hybrid_step(const tgs_param_ptrs* params, const tgs_param_ptrs* grads, const tgs_param_ptrs* m,
                           const tgs_param_ptrs* v, int64_t n, const uint8_t* touched, const float* view_rows,
                           int32_t k_rows, int32_t step, const int32_t* step_dev, const tgs_opt* opt,
                           void* workspace, size_t workspace_bytes, tgs_stream stream);

/*
 * Tile-error predictor (not in the paper): a 3-layer MLP 16 -> 128 -> 128 ->
 * 1 with ReLU that predicts log(1 + mean tile error) from per-tile features,
 * standing in for a dense refresh of stale error maps.  Weights are bfloat16
 * (bit patterns, row-major out x in: w1 [128,16], w2 [128,128], w3 [128]),
 * biases fp32; products accumulate in fp32.  Bias and weight updates run on
 * an fp32 master copy: a packed vector of tgs_mlp_param_count() floats laid
 * out as W1 | b1 | W2 | b2 | W3 | b3.
 */
typedef struct {
  const uint16_t* w1;
  const float* b1;
  const uint16_t* w2;
  const float* b2;
  const uint16_t* w3;
  const float* b3;
} tgs_mlp;

int32_t tgs_mlp_param_count(void);

/* y [R] = MLP(x [R,16] fp32, zero-padded features; rounded to bf16).  When
 * given, h1 and h2 [R,128] receive the bf16 hidden activations (post-ReLU)
 * for the backward. */
tgs_status tgs_mlp_forward(const tgs_mlp* w, int64_t rows, const float* x, float* y, uint16_t* h1, uint16_t* h2,
                           tgs_stream stream);

/* The same forward on the tcgen05 tensor cores (128-row tiles, operands in
 * shared memory, accumulators in tensor memory); x, w1, w2, h1, h2 16-byte
 * aligned.  status (nullable device int32) is set to 1 if a wait for the
 * tensor cores timed out (the call's outputs are then incomplete). */
tgs_status tgs_mlp_forward_tc(const tgs_mlp* w, int64_t rows, const float* x, float* y, uint16_t* h1, uint16_t* h2,
                              int32_t* status, tgs_stream stream);

/* Failure drill of the timeout path above (not in the paper): one CTA of the
 * same kernel allocates its tensor memory, waits a short bounded time on an
 * mbarrier phase that nothing completes, sets *status (device int32) to 1,
 * frees the tensor memory and returns.  No tensor-core work is issued. */
tgs_status tgs_mlp_tc_wait_drill(int32_t* status, tgs_stream stream);

/* Gradient of L = (1/R) sum (y - t)^2 / 2 into grads (packed layout, fp32,
 * overwritten) and *loss (device double), from the forward's x, h1, h2, y.
 * Hidden adjoints are rounded to bf16 before they meet a bf16 operand.  R is
 * rows, or min(rows, *rows_dev) when rows_dev (device int32) is given: the
 * rows past it are padding and take no part. */
size_t tgs_mlp_backward_workspace_size(int64_t rows);
tgs_status tgs_mlp_backward(const tgs_mlp* w, int64_t rows, const int32_t* rows_dev, const float* x,
                            const uint16_t* h1,
                            const uint16_t* h2, const float* y, const float* target, float* grads, double* loss,
                            void* workspace, size_t workspace_bytes, tgs_stream stream);

/* The same gradient on the tcgen05 tensor cores: the activation adjoint
 * dH1 = [H1 > 0] (dH2 W2) as one 128-row tile contraction per tile (operands
 * in shared memory, the accumulator in tensor memory), and the weight
 * gradients dW2 += dH2^T H1 and dW1 += dH1^T bf16(X) as contractions over 128-row tiles
 * (M = 128 hidden units, K = 128 rows), with the bias gradients as an extra
 * column of ones in the same contraction, accumulated in tensor memory per
 * CTA and added to grads once per CTA; dW3 and db3 on the CUDA cores.  The
 * products are the same bf16 x bf16 products with fp32 sums (the order of
 * the sums differs).  x, h1, h2 and the workspace 16-byte aligned.  status
 * (nullable device int32) is set to 1 if a wait for the tensor cores timed
 * out (grads are then incomplete). */
tgs_status tgs_mlp_backward_tc(const tgs_mlp* w, int64_t rows, const int32_t* rows_dev, const float* x,
                               const uint16_t* h1, const uint16_t* h2, const float* y, const float* target,
                               float* grads, double* loss, int32_t* status, void* workspace, size_t workspace_bytes,
                               tgs_stream stream);

/* One training pass on the tcgen05 tensor cores with the forward recomputed
 * in the same kernel: per 128-row tile the two hidden layers (as
 * tgs_mlp_forward_tc) and the gradient (as tgs_mlp_backward_tc), with the
 * activations kept on chip, so neither h1 nor h2 goes to memory.  Writes the
 * gradient of L = (1/R) sum (y - t)^2 / 2 into grads (packed layout, fp32,
 * overwritten) and L into *loss (device double); R as in tgs_mlp_backward.
 * y (nullable, [rows] fp32) receives the forward's outputs; they equal
 * tgs_mlp_forward_tc's up to the order of the sum over the hidden units.
 * x, w1 and w2 16-byte aligned.  status (nullable device int32) is set to 1
 * if a wait for the tensor cores timed out (grads are then incomplete). */
tgs_status tgs_mlp_train_tc(const tgs_mlp* w, int64_t rows, const int32_t* rows_dev, const float* x,
                            const float* target, float* y, float* grads, double* loss, int32_t* status,
                            tgs_stream stream);

/* Adam step on the fp32 master vector (params, m, v: tgs_mlp_param_count()
 * floats) with bias correction at `step` (>= 1); writes the bf16 copies of
 * W1, W2, W3. */
tgs_status tgs_mlp_adam(float* params, const float* grads, float* m, float* v, int32_t step, float lr,
                        float beta1, float beta2, float eps, uint16_t* w1, uint16_t* w2, uint16_t* w3,
                        tgs_stream stream);

/*
 * Tile memory and features of the tile-error predictor (not in the paper,
 * which refreshes a stale view's error map by rendering it, Sec. 3.3).
 *
 * tile_observe - after a step's loss: for each active rank j, the tile's
 * record mem[t] (float4: list length, mean T_final, mean err_pix over its
 * sampled pixels, 1 = observed) and mem_iter[t] = the iteration (iter_dev when
 * given); target[j] (nullable) = log(1 + mean err_pix), minus the same of the
 * tile's previous observation when residual = 1 and there was one; 0 for
 * ranks past n_active.  mem [T,4] (16-byte aligned), mem_iter [T]: the view's
 * memory, zero before the first observation.
 */
tgs_status tgs_tile_observe(const int32_t* active_tiles, const int32_t* n_active, int32_t n_active_max,
                            const int32_t* pix_off, const int32_t* tile_ranges, const float* T_final,
                            const float* err_pix, uint64_t iter, const uint64_t* iter_dev, float* mem,
                            int64_t* mem_iter, float* target, int32_t residual, tgs_stream stream);

/*
 * tile_features - x [n_rows_max, 16] (16-byte aligned) for tiles rows[r]
 * (r < *n_rows; zero rows after) or, with rows NULL, for every tile r <
 * n_rows_max: log(1 + list length), mean T_final (1 if never observed),
 * log(1 + error), view_cos (cosine between this view and a reference view
 * direction, from the host), log(1 + iterations since the observation;
 * 1e6 if never), cosine of the tile centre's ray to the optical axis, 1 if
 * observed; slots 7-15 zero.
 */
tgs_status tgs_tile_features(const float* mem, const int64_t* mem_iter, const int32_t* rows, const int32_t* n_rows,
                             int32_t n_rows_max, const tgs_camera* cam, float view_cos, uint64_t iter,
                             const uint64_t* iter_dev, float* x, tgs_stream stream);

/*
 * tile_refresh - rescales each tile of the fp16 error map [H,W] so that its
 * mean is exp(p) - 1, p = pred[t] (+ base[16 t + 2], the tile's last observed
 * log error from tile_features, when base is given: pred are then residuals),
 * clamped at 0 below, keeping the shape within the tile; a tile whose mean
 * is 0 is set to the prediction everywhere.
 */
tgs_status tgs_tile_refresh(const float* pred, const float* base, uint16_t* err_map, int32_t width, int32_t height,
                            tgs_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* TURBOGS_H */
