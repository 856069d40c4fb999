/* gs.h -- C ABI of the GB300 (sm_103a) differentiable Gaussian-splatting rasterizer.
 *
 * The library renders RGB, depth, alpha and an n_feat-channel feature map of a set of
 * 3D Gaussians seen by a pinhole camera, and back-propagates into every Gaussian
 * parameter and the 6-DoF camera pose.  It implements the rasterizer under the X-GS
 * Perceiver (arxiv 2603.09632):
 *   - Gaussians Theta = {mu, Sigma, alpha, c} with Sigma = R S S^T R^T   (App. A)
 *   - EWA projection Sigma' = J W Sigma W^T J^T                          (App. A)
 *   - front-to-back blending C = sum_i c_i a'_i prod_{j<i}(1 - a'_j)     (Eq. 1, App. B)
 *   - depth by substituting c_i -> d_i (App. B), features c_i -> f_i (Sec. 3.1)
 *   - gradients for mapping (Eq. 3) and tracking (Eq. 2, App. B)
 *
 * Conventions (all inputs are plain pointers; no PyTorch types cross this boundary):
 *   - Pointers named "device" must point to memory on the workspace's device.  The
 *     caller owns every input and output buffer; the library owns the workspace.
 *   - Inputs are post-activation: scales > 0, opacities in [0,1], quaternions (w,x,y,z)
 *     non-zero and not necessarily unit (they are normalised inside).
 *   - Camera: OpenCV axes (x right, y down, z forward); R (row-major) and t map world to
 *     camera; pixel (x, y) is sampled at its centre (x + 0.5, y + 0.5); Gaussians with
 *     camera-space depth <= near_z are culled.  Tiles are 16 x 16 pixels.
 *   - Image outputs are float32, channel-major: rgb[3][H][W], depth[H][W], alpha[H][W],
 *     feat[n_feat][H][W].  Any output pointer may be NULL (not written).
 *   - Every call is asynchronous on the given CUDA stream (a cudaStream_t passed as
 *     void*; NULL = legacy default stream) unless its comment says it synchronises.
 *   - Errors are returned, never thrown or aborted.  Errors that kernels detect (an
 *     instance count above the reserved capacity in the no-sync path) set a device status
 *     word; gs_workspace_status() reads and clears it.
 *   - Calls on one workspace must be issued from one host thread at a time and kept in
 *     stream order: gs_project -> gs_bin_tiles -> gs_render_fwd -> gs_render_bwd.
 */
#ifndef GS_H_
#define GS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GS_OK = 0,
  GS_ERR_ARG = 1,          /* invalid argument (null pointer, size, unsupported option) */
  GS_ERR_OOM = 2,          /* device allocation failed */
  GS_ERR_CUDA = 3,         /* a CUDA runtime call failed */
  GS_ERR_DEVICE = 4,       /* a kernel reported an error through the device status word */
  GS_ERR_TIMEOUT = 5,      /* a bounded wait expired */
  GS_ERR_BUSY = 6,         /* request not finished yet (serving poll) */
  GS_ERR_OVER_BUDGET = 7,  /* request cannot fit the serving memory budget */
  GS_ERR_STATE = 8,        /* calls out of order (e.g. render before project/bin) */
  GS_ERR_CANCELLED = 9     /* serving request cancelled before it started */
} gs_status;

typedef enum { GS_F32 = 0, GS_BF16 = 1 } gs_dtype;

/* Pinhole camera (App. A: "viewing transformation W" and the Jacobian J of the
 * projection).  cx, cy are free; the synthetic workloads use W/2, H/2.
 * stride/off_x/off_y select grid-sampled rendering (Sec. 3.2 and App. D, "Dynamic Grid
 * Sampling"): stride 1 with offsets 0 renders every pixel.  With stride s (1..256) and
 * offsets 0 <= off_x, off_y < s the renderer computes only the samples (m, n) of the
 * compact Hs x Ws grid, Hs = ceil(H / s), Ws = ceil(W / s), sample (m, n) being image pixel
 * (row off_y + m s, column off_x + n s); every image output and upstream gradient of
 * gs_render_fwd / gs_render_bwd is then a compact [.., Hs, Ws] map.  Each sample equals the
 * full-resolution render at its pixel; samples beyond the image (large offsets) render
 * nothing (alpha 0, zero colour, depth and features).  Other values: GS_ERR_ARG. */
typedef struct {
  int32_t W, H;
  float fx, fy, cx, cy;
  float R[9];     /* world -> camera rotation, row-major */
  float t[3];     /* world -> camera translation */
  float near_z;   /* near-plane depth, > 0 (0.2 in the workloads) */
  int32_t tile;   /* must be 16 */
  int32_t stride, off_x, off_y;
} gs_camera;

/* Scene (App. A parameter set Theta plus the per-Gaussian feature vector f_i of Sec. 3.1).
 * All arrays are device pointers, row-major, 16-byte aligned. */
typedef struct {
  int64_t n;              /* number of Gaussians, 0 <= n < 2^31 */
  int32_t sh_degree;      /* 0..3; K = (sh_degree+1)^2 coefficients per colour channel */
  int32_t n_feat;         /* 0..64 feature channels */
  int32_t feat_dtype;     /* gs_dtype of feats */
  const float* means;     /* [n][3] world positions */
  const float* scales;    /* [n][3] > 0 */
  const float* quats;     /* [n][4] (w, x, y, z) */
  const float* opacities; /* [n] in [0, 1] */
  const float* sh;        /* [n][K][3] real SH coefficients, (l, m = -l..l) order */
  const void* feats;      /* [n][n_feat] float32 or bfloat16 */
} gs_scene;

typedef struct gs_workspace gs_workspace;

/* Counts of the last projection/binning and forward render (for roofline accounting). */
typedef struct {
  int64_t n;            /* Gaussians */
  int64_t visible;      /* V: Gaussians with a non-empty tile rectangle */
  int64_t instances;    /* I: (tile, Gaussian) pairs */
  int64_t inst_eff;     /* I_eff: sum over tiles of the longest list prefix a pixel used */
  int64_t pixels;       /* P */
  int64_t tiles;        /* T */
  int64_t pairs_eval;   /* sum over pixels of the list entries up to the last contributor */
  int64_t pairs_blend;  /* sum over pixels of the Gaussians actually blended */
} gs_stats;

/* Human-readable name of a status code (static string). */
const char* gs_status_string(gs_status s);

/* Create a workspace bound to CUDA device `device`.  *ws receives the handle.
 * Errors: GS_ERR_ARG (ws NULL), GS_ERR_CUDA (bad device). */
gs_status gs_workspace_create(gs_workspace** ws, int device);

/* Free the workspace and all its device memory (synchronises the device).  NULL is a
 * no-op. */
void gs_workspace_destroy(gs_workspace* ws);

/* Pre-allocate capacity for n_gauss Gaussians, n_instances tile instances, n_pixels pixels
 * and n_feat channels, so that later calls allocate nothing (required for the no-sync
 * path of gs_bin_tiles and for CUDA-graph capture).  Synchronous.  Errors: GS_ERR_OOM. */
gs_status gs_workspace_reserve(gs_workspace* ws, int64_t n_gauss, int64_t n_instances,
                               int64_t n_pixels);

/* Synchronise `stream`, read and clear the device status word.  Returns GS_OK or
 * GS_ERR_DEVICE (e.g. the instance count exceeded the reserved capacity).
 * Errors: GS_ERR_ARG (NULL workspace), GS_ERR_CUDA. */
gs_status gs_workspace_status(gs_workspace* ws, void* stream);

/* Device memory held by the workspace, in bytes, into *bytes (host pointer): the sum of
 * its buffers' capacities, i.e. its high-water mark, since buffers only grow.  No device
 * work.  Errors: GS_ERR_ARG (null argument). */
gs_status gs_workspace_bytes(gs_workspace* ws, int64_t* bytes);

/* a1. EWA projection and SH colour, one thread per Gaussian (App. A, Sigma and Sigma';
 * SH colour along the view direction from the camera centre).  Writes, into the
 * workspace, each Gaussian's 2D mean, conic (inverse of Sigma' + 0.3 I), depth, colour,
 * tile rectangle (3-sigma bound) and tile count.  Culled Gaussians (depth <= near_z,
 * degenerate Sigma', empty rectangle) get no tiles.  Grows the workspace if needed.
 * Errors: GS_ERR_ARG for a NULL scene, camera or workspace, n outside [0, 2^31), sh_degree
 * outside [0, 3], n_feat outside [0, 64], an unknown feat_dtype, a missing or not
 * 16-byte-aligned parameter array, a camera with W or H <= 0 (or above 65535 tiles), a
 * tile size other than 16, fx, fy or near_z not > 0, or a stride outside [1, 256] or
 * offsets outside [0, stride); GS_ERR_OOM if the workspace cannot grow; GS_ERR_CUDA. */
gs_status gs_project(const gs_scene* scene, const gs_camera* cam, gs_workspace* ws,
                     void* stream);

/* a2. Tile/depth binning ("depth-sorted", Eq. 1).  Produces, per 16x16 tile, the list
 * of Gaussians covering it sorted by (depth, id), in tile buckets: the per-tile instance
 * counts (added by gs_project) are scanned into tile ranges, the instances are scattered
 * into their tiles' ranges, and each range is sorted by depth with a hand-written LSD
 * radix sort, equal depths in id order.  Calling it again before the next gs_project
 * changes nothing.
 * If n_instances_out is non-NULL the call synchronises the stream once to read the
 * instance count I, grows the workspace if needed and stores I there.  If it is NULL
 * the call never synchronises: the reserved instance capacity must be large enough,
 * otherwise the excess is dropped and the device status word records the overflow.
 * Errors: GS_ERR_ARG (NULL workspace), GS_ERR_STATE (no gs_project before it), GS_ERR_OOM
 * (the instance buffers cannot grow), GS_ERR_CUDA. */
gs_status gs_bin_tiles(gs_workspace* ws, int64_t* n_instances_out, void* stream);

/* a3. Forward rendering (Eq. 1 front-to-back alpha blending; depth, App. B; features,
 * Sec. 3.1), one CTA per tile.  Blending skips a Gaussian with alpha < 1/255, caps alpha
 * at 0.99 and stops before a Gaussian that would take transmittance below 1e-4;
 * alpha = 1 - T_final.  Outputs are device pointers (see conventions), any may be NULL.
 * The per-pixel final transmittance and contributor count are kept for gs_render_bwd.
 * scene and cam must be those given to gs_project.
 * Errors: GS_ERR_ARG as gs_project, and for a feat pointer that is not 16-byte aligned;
 * GS_ERR_STATE if the workspace holds no binned projection of a scene of this size with
 * this camera grid; GS_ERR_CUDA. */
gs_status gs_render_fwd(const gs_scene* scene, const gs_camera* cam, gs_workspace* ws,
                        float* rgb, float* depth, float* alpha, float* feat, void* stream);

/* Masked L1 + cosine feature loss of App. D ("Masked Loss Evaluation"), evaluated on the
 * rendered feature map G_hat (n_feat x rows x cols of the camera's grid, P samples) in
 * the forward's epilogue.  With a = V G_hat and b = V G* per sample:
 *   L_1 = sum |a - b| / (n_feat P),   L_cos = sum_p (1 - cos(a_p, b_p)) / P,
 *   cos(a, b) = a.b / (max(|a|, 1e-8) max(|b|, 1e-8)),   L = lambda_sem (L_cos + L_1);
 * masked samples add the constant 1 to L_cos's sum and no gradient. */
typedef struct {
  const float* target;   /* G* [n_feat][rows][cols], device (e.g. from gs_grid_target_*) */
  const float* mask;     /* V [rows][cols] (0/1), device; NULL = all ones */
  float lambda_sem;      /* weight, >= 0 */
  float* g_feat;         /* out: dL/dG_hat [n_feat][rows][cols], device; pass it to
                            gs_render_bwd as g_feat */
  double* loss;          /* out: [3] = (L, L_1, L_cos), device; overwritten */
} gs_feat_loss;

/* NEXT-2: gs_render_fwd with the feature loss fused into its epilogue: the loss value and
 * its gradient dL/dG_hat are produced without writing G_hat (feat may be NULL) or running
 * a separate loss pass.  Requires n_feat > 0.  Errors as gs_render_fwd; GS_ERR_ARG for a
 * NULL loss, target, g_feat or loss pointer or a negative lambda_sem. */
gs_status gs_render_fwd_loss(const gs_scene* scene, const gs_camera* cam, gs_workspace* ws,
                             float* rgb, float* depth, float* alpha, float* feat,
                             const gs_feat_loss* loss, void* stream);

/* a4 + a5. Backward of gs_render_fwd (App. B: the rasterizer is differentiable; Eq. 2
 * tracking, Eq. 3 mapping).  Inputs are the upstream gradients of the four images (device,
 * same layout as the outputs; NULL = zero).  Outputs (device, overwritten, zero for culled
 * Gaussians): g_means [n][3], g_scales [n][3], g_quats [n][4] (w.r.t. the raw quaternion),
 * g_opac [n], g_sh [n][K][3], g_feats [n][n_feat] (float32 whatever feat_dtype is), and
 * g_pose6 [6] = dL/dxi of the left twist perturbation T <- Exp(xi) T, xi = (rho, phi).
 * Any output may be NULL (not written).  Must follow gs_render_fwd on the same
 * workspace with the same scene and camera.
 * Errors: GS_ERR_ARG as gs_project, and for g_feats or g_quats not 16-byte aligned;
 * GS_ERR_STATE if no gs_render_fwd of a scene of this size with this camera grid precedes
 * it on the workspace; GS_ERR_CUDA. */
gs_status gs_render_bwd(const gs_scene* scene, const gs_camera* cam, gs_workspace* ws,
                        const float* g_rgb, const float* g_depth, const float* g_alpha,
                        const float* g_feat, float* g_means, float* g_scales, float* g_quats,
                        float* g_opac, float* g_sh, float* g_feats, float* g_pose6,
                        void* stream);

/* Upstream gradient of the L1 loss scale * sum|pred - target| (the distillation loss of
 * the semantic workload): grad = scale * sign(pred - target), 0 where equal.  Device
 * pointers, n elements.  May alias grad == pred.
 * Errors: GS_ERR_ARG (n < 0, or a NULL pointer with n > 0), GS_ERR_CUDA. */
gs_status gs_l1_grad(const float* pred, const float* target, int64_t n, float scale,
                     float* grad, void* stream);

/* ---- grid-sampled supervision targets (Sec. 3.2; App. D, "Compact Predictions and
 * Targets") ------------------------------------------------------------------------
 * Both fill the compact target G* [D][Hs][Ws] and the validity mask V [Hs][Ws] (floats
 * 0 / 1; mask may be NULL) of the stride-s sample grid with offsets (off_x, off_y):
 * Hs = ceil(H / s), Ws = ceil(W / s), sample (m, n) = image pixel (row off_y + m s,
 * column off_x + n s), the grid gs_render_fwd draws for the same camera fields.  Samples
 * beyond the image get V = 0 and zero targets.  All pointers are caller-owned device
 * memory; the calls are asynchronous on `stream`.  Errors: GS_ERR_ARG for non-positive
 * sizes, a stride outside 1..256 or an offset outside [0, stride). */

/* Region-indexed annotations: seg [H][W] int32 region ids (-1 = background) and a
 * region-feature table [R][D].  V = 1 where the sampled id lies in [0, R), and G* is that
 * table row; any other id counts as background (V = 0, G* = 0).
 * Errors: GS_ERR_ARG (grid arguments as in gs_camera, R or D < 0, or a NULL seg, table or
 * target where needed), GS_ERR_CUDA. */
gs_status gs_grid_target_region(const int32_t* seg, int32_t H, int32_t W, const float* table,
                                int32_t R, int32_t D, int32_t stride, int32_t off_x, int32_t off_y,
                                float* target, float* mask, void* stream);

/* Continuous feature map fmap [D][Hf][Wf] at a lower resolution: sample (u, v) reads the
 * map at (round(u (Hf - 1) / max(H - 1, 1)), round(v (Wf - 1) / max(W - 1, 1))), halves
 * rounded away from zero (exact integer arithmetic); V = 1 inside the image.
 * Errors: GS_ERR_ARG (grid arguments as in gs_camera, D < 0, Hf or Wf <= 0, or a NULL fmap
 * or target with D > 0), GS_ERR_CUDA. */
gs_status gs_grid_target_resample(const float* fmap, int32_t D, int32_t Hf, int32_t Wf, int32_t H,
                                  int32_t W, int32_t stride, int32_t off_x, int32_t off_y,
                                  float* target, float* mask, void* stream);

/* ---- VQ semantic parameterisation and decode (NEXT-4; Sec. 3.2 "Online VQ Module",
 * App. E) ---------------------------------------------------------------------------
 * Each Gaussian carries logits z_i [L] over a shared codebook E [L][D]; the renderer
 * splats the mixture weights w_i = softmax(z_i) through the feature path (n_feat = L,
 * feats = the weights), and a pixel's semantic feature is F(x) = E^T w(x). */

/* w = softmax(z) per Gaussian: logits [n][L] float32 (device) -> w_out [n][L] of
 * out_dtype (GS_BF16 to render them as bf16 features, or GS_F32).  1 <= L <= 64.
 * Errors: GS_ERR_ARG. */
gs_status gs_vq_weights(const float* logits, int64_t n, int32_t L, int32_t out_dtype, void* w_out,
                        void* stream);

/* Backward of gs_vq_weights: g_logits = w * (g_w - sum_l g_w,l w_l), w recomputed from the
 * logits.  All [n][L] float32 device arrays.
 * Errors: GS_ERR_ARG (n < 0, L outside [1, 64], or a NULL array with n > 0), GS_ERR_CUDA. */
gs_status gs_vq_weights_bwd(const float* logits, const float* g_w, int64_t n, int32_t L,
                            float* g_logits, void* stream);

/* Decode of a rendered weight map on the tensor cores (tcgen05; FP32-accurate products by
 * the 3xTF32 split of both operands, FP32 accumulation; above 256 columns a cluster of two
 * CTAs on two SMs, each with half of the columns): wmap [L][P] float32 (the channel-major feature output of a render with
 * the weights as features, P pixels), codebook [L][D] float32.  Writes, when non-NULL:
 *   F_out [D][P] = E^T w(x) per pixel;
 *   relevance [P] = max_{n >= 1} 1 / (1 + exp(tau (F~.t_n - F~.t_0))), F~ = F / (|F| + 1e-8),
 *     the prompt relevance of App. E with text [n_text][D] (row 0 the prompt, rows 1.. the
 *     negatives, unit vectors; 2 <= n_text <= 8) and tau = 10 in the paper.
 * L a multiple of 8 in [8, 64]; D a multiple of 16 in [16, 512].  err (device int32, may be
 * NULL) is set to 1 if a tensor-core completion wait timed out (outputs then invalid).
 * Accuracy: |F - E^T w| <= 2e-5 sum_l |w_l E_l| per entry (products to 2^-22, FP32 sums).
 * Errors: GS_ERR_ARG for unsupported sizes or missing pointers. */
gs_status gs_vq_decode(const float* wmap, int64_t P, int32_t L, const float* codebook, int32_t D,
                       float* F_out, const float* text, int32_t n_text, float tau,
                       float* relevance, int32_t* err, void* stream);

/* ---- introspection (synchronous; host pointers) ---------------------------------- */

/* Counts of the last gs_project/gs_bin_tiles/gs_render_fwd.  inst_eff is computed by a
 * small reduction over the per-pixel contributor counts.  Synchronises `stream`.
 * Errors: GS_ERR_ARG (NULL argument), GS_ERR_OOM, GS_ERR_CUDA. */
gs_status gs_get_stats(gs_workspace* ws, gs_stats* out, void* stream);

/* Copy the sorted instance list to host: tile id and Gaussian id per instance, at most
 * cap entries; *n_out receives I.  ranges_out (may be NULL) receives 2*T uint32
 * [start, end) per tile.  Synchronises `stream`.
 * Errors: GS_ERR_ARG (NULL workspace, cap < 0), GS_ERR_STATE (nothing binned yet),
 * GS_ERR_CUDA. */
gs_status gs_get_instances(gs_workspace* ws, uint32_t* tiles_out, uint32_t* ids_out,
                           int64_t cap, int64_t* n_out, uint32_t* ranges_out, void* stream);

/* Copy the projection of the last gs_project to host (arrays of n entries; any NULL):
 * mean2d [n][2], conic [n][3], depth [n], rgb [n][3], rect [n][4] = (x0, y0, x1, y1)
 * tiles, all zero for culled Gaussians.  Synchronises `stream`.
 * Errors: GS_ERR_ARG (NULL workspace), GS_ERR_STATE (no gs_project yet), GS_ERR_CUDA. */
gs_status gs_get_projection(gs_workspace* ws, float* mean2d, float* conic, float* depth,
                            float* rgb, int32_t* rect, void* stream);

/* Copy the per-pixel final transmittance and contributor count of the last forward
 * render to host ([H][W] each; either may be NULL).  Synchronises `stream`.
 * Errors: GS_ERR_ARG (NULL workspace), GS_ERR_STATE (no render yet), GS_ERR_CUDA. */
gs_status gs_get_pixel_state(gs_workspace* ws, float* T_final, uint32_t* n_contrib,
                             void* stream);

/* ---- stage timing (CUDA events on the launching stream) ---------------------------- */

enum { GS_TIMER_PROJECT = 0, GS_TIMER_BIN = 1, GS_TIMER_FWD = 2, GS_TIMER_BWD_RASTER = 3,
       GS_TIMER_BWD_PROJECT = 4, GS_NUM_TIMERS = 5 };

/* Enable (1) or disable (0) event timing of the stages above.  While enabled, each stage
 * records a CUDA event pair around its kernels on the caller's stream.
 * Errors: GS_ERR_ARG (NULL workspace), GS_ERR_CUDA (event creation). */
gs_status gs_timing_enable(gs_workspace* ws, int enable);

/* Synchronise, add up the elapsed times of all recorded event pairs and reset them.
 * ms_out[GS_NUM_TIMERS] receives total milliseconds, count_out[GS_NUM_TIMERS] (may be
 * NULL) the number of timed launches of each stage.
 * Errors: GS_ERR_ARG (NULL workspace or ms_out), GS_ERR_CUDA. */
gs_status gs_timing_collect(gs_workspace* ws, double* ms_out, int64_t* count_out);

/* Number of CUDA kernels this library has launched in the process so far (all
 * workspaces, all devices).  Host-side counter; no synchronisation. */
int64_t gs_launch_count(void);

/* FP32 arithmetic peak of the current device, measured: not a step of the paper's method
 * but the denominator of the rasterizer's roofline (blending, Eq. 1, and its backward,
 * App. B, are bound by FP32 arithmetic).  Launches two kernels that fill every SM to its
 * occupancy limit with threads advancing eight independent fused multiply-add chains for
 * `iters` x 16 steps each, one with scalar FMAs and one with packed pairs (two FMAs per
 * instruction), each after a short warm-up launch; times them with CUDA events on
 * `stream` and synchronises on the end events.  *tflops_out receives the larger FP32 rate
 * (2 FLOPs per FMA), *ms_out (may be NULL) that kernel's time.  Reads and changes no GPU
 * setting; the caller samples the SM clock if it wants the rate at a known clock.
 * Errors: GS_ERR_ARG (iters <= 0, NULL tflops_out), GS_ERR_CUDA. */
gs_status gs_measure_fp32_peak(int iters, double* tflops_out, double* ms_out, void* stream);

/* ---- serving ----------------------------------------------------------------------
 *
 * Keeps several scenes resident on one GPU and renders requests (forward, optionally
 * backward) with continuous batching.  The Perceiver renders many views of the same map
 * (tracking, mapping over a keyframe window, semantic phases; Sec. 3.2, Eq. 2-3); serving
 * is the systems form of that load.
 *   - Memory.  At the first submit the server divides its budget once: resident scenes,
 *     then request workspaces (min(4, max_slots) lanes of ceil(max_slots / lanes)
 *     workspaces, reserved for the largest scene and a per-request pixel limit; together at
 *     most half of what the scenes leave), then one arena of tile-instance buffers with the
 *     rest.  Nothing is
 *     allocated or freed while requests run, and scenes can no longer be added.
 *   - Admission in two phases.  Each lane is a worker that takes a batch of the oldest
 *     pending requests (one per workspace) and projects them; each request's tile-instance count (read back once per
 *     batch) is what it needs from the arena.  Ranges are granted in arrival order; a
 *     request that does not fit waits at the head of the queue, and once it has waited
 *     50 ms no request behind it is admitted before it.
 *   - Execution.  The admitted requests are binned into their ranges and rendered by ONE
 *     persistent forward raster launch whose queue holds every (request, tile) item of the
 *     batch (one launch per feature layout), then one backward raster launch for those
 *     that want gradients and their projection backward.  Lanes run independently, so
 *     while one lane's batch is on the device the others admit and launch theirs:
 *     requests that arrive meanwhile start as a lane and memory free up, and their work
 *     overlaps on the device.
 * A request's results equal those of the same request rendered alone (forward bit for
 * bit; backward up to the order of atomic additions).  Host-side waits are bounded by the
 * caller's timeout; no kernel waits on another. */
typedef struct gs_server gs_server;

typedef struct {
  int32_t scene_id;       /* from gs_serve_add_scene */
  gs_camera cam;
  int32_t want_bwd;       /* 1: also run gs_render_bwd */
  /* caller-owned device outputs, as for gs_render_fwd (any may be NULL) */
  float *rgb, *depth, *alpha, *feat;
  /* when want_bwd: upstream gradients and gradient outputs, as for gs_render_bwd */
  const float *g_rgb, *g_depth, *g_alpha, *g_feat;
  float *g_means, *g_scales, *g_quats, *g_opac, *g_sh, *g_feats, *g_pose6;
} gs_request;

typedef struct {
  gs_status status;       /* outcome of the request */
  int32_t slot;           /* workspace that ran it: lane x slots per lane + slot (-1: never) */
  int64_t instances;      /* tile instances of its binning */
  double queue_us;        /* submit -> start */
  double run_us;          /* start -> results ready on the device */
  double latency_us;      /* submit -> results ready */
} gs_result;

/* Create a server on `device` with a device-memory budget (bytes) for everything it holds
 * (resident scenes, request workspaces, the instance arena) and max_slots (1..64): up to
 * ceil(max_slots / lanes) (at most 8) requests per batch on each of min(4, max_slots)
 * lanes.  Nothing is
 * allocated on the device until scenes are added.  Errors: GS_ERR_ARG, GS_ERR_CUDA. */
gs_status gs_serve_create(gs_server** server, int device, int64_t hbm_budget_bytes, int max_slots);

/* Cancel pending requests, wait for running ones, free everything.  NULL is a no-op. */
void gs_serve_destroy(gs_server* server);

/* Copy a scene (device pointers, as for gs_project) into server-owned device memory.
 * *scene_id receives its id.  GS_ERR_OVER_BUDGET if it does not fit the budget;
 * GS_ERR_STATE once a request has been submitted (the budget is divided then);
 * GS_ERR_ARG, GS_ERR_OOM. */
gs_status gs_serve_add_scene(gs_server* server, const gs_scene* scene, int* scene_id);

/* Queue a request; *ticket identifies it.  The request struct is copied; its buffers
 * must stay valid until the request is polled.  The first submit divides the budget
 * (see above) and may allocate.  GS_ERR_OVER_BUDGET if the image exceeds the per-request
 * pixel limit or the budget cannot hold the workspaces; GS_ERR_ARG for an unknown scene
 * or a bad camera (grid sampling is not served).  A request whose tile instances exceed
 * the whole arena finishes with status GS_ERR_OVER_BUDGET. */
gs_status gs_serve_submit(gs_server* server, const gs_request* req, uint64_t* ticket);

/* Wait up to timeout_us (0: do not wait; negative: wait without limit) for a request.
 * GS_OK with *result filled (result->status is the request's own outcome) and the
 * ticket released; GS_ERR_BUSY if not finished in time; GS_ERR_ARG for an unknown or
 * already released ticket. */
gs_status gs_serve_poll(gs_server* server, uint64_t ticket, int64_t timeout_us, gs_result* result);

/* Cancel a request that is waiting in the queue (its result status becomes
 * GS_ERR_CANCELLED); GS_ERR_BUSY once a batch has taken it; GS_ERR_ARG for an unknown
 * ticket or a server that has no request yet. */
gs_status gs_serve_cancel(gs_server* server, uint64_t ticket);

/* Memory held by resident scenes, arena bytes granted to the requests running now and
 * its peak, and the peak number of requests running at once (any may be NULL).
 * Errors: GS_ERR_ARG (NULL server). */
gs_status gs_serve_info(gs_server* server, int64_t* scene_bytes, int64_t* in_flight_bytes,
                        int64_t* peak_in_flight_bytes, int32_t* peak_running);

typedef struct {
  int64_t scene_bytes;       /* resident scenes */
  int64_t workspace_bytes;   /* request workspaces and queues, reserved at the first submit */
  int64_t arena_bytes;       /* tile-instance arena */
  int64_t arena_peak_bytes;  /* most of it granted at once */
  int64_t max_pixels;        /* per-request pixel limit */
  int64_t batches;           /* batches launched */
  int32_t lanes, slots_per_lane, peak_batch, peak_running;
} gs_serve_stats_t;

/* How the server divided its budget and how it batched: fills *out (zeros before the
 * first submit).  Errors: GS_ERR_ARG (NULL server or out). */
gs_status gs_serve_stats(gs_server* server, gs_serve_stats_t* out);

/* ---- rendering without allocation ------------------------------------------------
 *
 * gs_render_fwd_noalloc renders like gs_project -> gs_bin_tiles -> gs_render_fwd (same
 * kernels, same images) but allocates nothing: no workspace, no cudaMalloc, no
 * allocating library call.  It serves callers that cannot allocate device memory when
 * they render -- a plugin inside a host application that owns every allocation, code
 * held to a fixed device-memory budget, or a context where a cudaMalloc would stall or
 * fail.  The paper has no counterpart; this is an interface convenience.
 *
 * Every intermediate buffer lives in one file-scope device array of about 4 MB that
 * each device using the library holds until the process exits.  That bounds the
 * request: at most 16384 Gaussians, 131072 tile instances, 65536 pixels and 1024 tiles
 * (e.g. 256 x 256); a larger request returns GS_ERR_OVER_BUDGET and writes no output (the
 * instance limit is only known after projection, so that refusal comes after one
 * projection kernel has run on `stream`).
 *   - The first call on a device, with that device current, looks the array's device
 *     address up with cudaGetSymbolAddress (once per device); make that first call
 *     before any stream capture.
 *   - Every call on a device shares the array and it keeps the last call's contents:
 *     every call first clears, on `stream`, what must start at zero (its counters, its
 *     persistent-kernel queues and the tile counts of its image).  Calls that overlap on
 *     the GPU (other streams, other threads) race on the array and must be serialised by
 *     the caller.
 *   - Every call synchronises `stream` once, after projection, to read the instance
 *     count it checks against the limit.
 * scene, cam and the outputs are as for gs_project / gs_render_fwd (device pointers,
 * outputs channel-major, any output may be NULL).  Errors: GS_ERR_ARG, GS_ERR_OVER_BUDGET,
 * GS_ERR_CUDA. */
gs_status gs_render_fwd_noalloc(const gs_scene* scene, const gs_camera* cam, float* rgb,
                                float* depth, float* alpha, float* feat, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GS_H_ */
