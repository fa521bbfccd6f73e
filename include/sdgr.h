/*
 * sdgr.h -- C ABI of the B300 (sm_103a) SAR Differentiable Gaussian
 * Rasterizer (SDGR) of SAR-GS (arXiv 2506.21633).
 *
 * Problem statement (Section II, Fig. "SARGSflow"): scene Gaussians plus
 * radar geometry (azimuth angle, grazing angle, range / azimuth resolution)
 * in; SAR intensity images and the gradients of an image loss with respect
 * to every Gaussian parameter out.
 *
 * Conventions shared by every call
 *  - Pointers named "device" are CUDA device pointers on the current device;
 *    pointers named "host" are host memory.  The library never allocates
 *    device memory: the caller allocates every device buffer, including the
 *    workspace of sdgr_workspace_size() bytes, and owns it.  Host memory the
 *    library needs for its own bookkeeping is allocated in sdgr_ws_create()
 *    and freed in sdgr_ws_destroy().
 *  - Every compute call enqueues work on `stream` (a cudaStream_t; NULL =
 *    the legacy default stream) and returns without waiting for it.  No
 *    compute call synchronises the host, so a sequence of them can be
 *    captured into a CUDA graph.
 *  - Return codes report host-side validation and launch errors.  Conditions
 *    only the device can see (instance capacity exceeded) are written to the
 *    workspace's status word and read back with sdgr_read_status() once the
 *    stream has finished.  No call aborts, traps or prints.
 *  - Gaussian parameters, float32, row-major [N][12] (three float4 per
 *    Gaussian, 16-byte aligned):
 *        { mu_x, mu_y, mu_z, opacity_logit },
 *        { log_s_x, log_s_y, log_s_z, P },
 *        { q_w, q_x, q_y, q_z }
 *    mu = mean (world metres), s = exp(log_s) the axis scales, q an
 *    unnormalised rotation quaternion (Sigma = R(q/|q|) diag(s^2) R^T,
 *    eq. G(x)), opacity o = sigmoid(opacity_logit) standing for the two-way
 *    extinction 1 - E+ E- of eq. I_i, P the scattering coefficient.
 *    Gradients use the same layout.
 *  - Images: float32, one NR x NA block per view, views concatenated in view
 *    order; row = slant-range bin (near range first), column = azimuth bin;
 *    pixel (m, n) has its centre at pixel coordinates (m, n).
 */
#ifndef SDGR_H
#define SDGR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SDGR_OK = 0,
    SDGR_ERR_INVALID = 1,  /* an argument failed host-side validation */
    SDGR_ERR_CUDA = 2,     /* a CUDA runtime call or launch failed */
    SDGR_ERR_CAPACITY = 3, /* instance capacity exceeded (device status) */
    SDGR_ERR_TIMEOUT = 4,  /* a bounded device wait gave up (device status) */
    SDGR_ERR_STATE = 5,    /* calls made out of order on a workspace */
    SDGR_ERR_BOUNDS = 6    /* checked build only: an index left its buffer (device status) */
} sdgr_status;

/* One radar view (Section II-A-1, eqs. W and R_r).
 * phi   radar azimuth angle (rad); theta grazing angle (rad), 0 < theta < pi/2
 * dA    azimuth pixel size (m) > 0;  dR slant-range pixel size (m) > 0
 * NA    image columns (azimuth) > 0; NR image rows (slant range) > 0
 * scene index of the scene (a contiguous range of Gaussians) this view sees
 * center the world point the beam is centred on (m); it maps to the image
 *        centre, pixel coordinates (NA/2 - 1/2, NR/2 - 1/2). */
typedef struct {
    double phi, theta;
    double dA, dR;
    int32_t NA, NR;
    int32_t scene, reserved;
    double center[3];
} sdgr_view;

/* Renderer options (readings of passages the paper leaves open).
 * cutoff_K      contributions with Mahalanobis distance > K are zero on both
 *               planes (default 5)
 * dilation_eps  added to both 2D covariances, px^2 (default 0.3)
 * T_min         a ray stops once its transmittance drops below T_min
 *               (default 0: never; values below 2^-100 act as 2^-100, where
 *               the remaining contributions are below float32 resolution)
 * norm_mode     0: beta = exp(-delta/2) / (2 pi sqrt(det Sigma'_I)), so a
 *               Gaussian deposits its intensity in the image (default);
 *               1: beta = exp(-delta/2) (peak-normalised)
 * alpha_mode    opacity of Gaussian i on a ray where its profile
 *               exp(-delta/2) is G (attenuation factor of eq. I_i):
 *               0: alpha = o G, o = sigmoid(opacity logit) (default);
 *               1: alpha = 1 - exp(-tau G), tau = softplus(opacity logit)
 *               (Beer-Lambert; the peak opacity is again sigmoid(logit)) */
typedef struct {
    float cutoff_K;
    float dilation_eps;
    float T_min;
    int32_t norm_mode;
    int32_t alpha_mode;
} sdgr_cfg;

/* Workspace capacities.  A workspace created for these capacities accepts
 * any call whose totals do not exceed them.
 * max_views       number of views per call
 * max_scenes      number of scenes per call
 * max_gaussians   total Gaussians over all scenes
 * max_view_gauss  sum over views of the Gaussian count of the view's scene
 * max_pixels      sum over views of NA * NR
 * max_tiles       sum over views of ceil(NA/16) * ceil(NR/16)
 * max_instances   (tile, Gaussian) pairs over both planes of all views */
typedef struct {
    int32_t max_views;
    int32_t max_scenes;
    int64_t max_gaussians;
    int64_t max_view_gauss;
    int64_t max_pixels;
    int64_t max_tiles;
    int64_t max_instances;
} sdgr_caps;

/* Opaque workspace handle: host-side plan plus the caller's device buffer. */
typedef struct sdgr_ws sdgr_ws;

/* Capacities that exactly fit one call (host only, no CUDA call).
 * scene_offsets: host, n_scenes + 1 increasing entries; scene s owns
 * Gaussians [scene_offsets[s], scene_offsets[s+1]).  instances: the
 * max_instances to reserve (>= 0; see sdgr_read_status for the exact need).
 * Returns SDGR_ERR_INVALID on a malformed view or scene table. */
sdgr_status sdgr_caps_for(const sdgr_view *views, int32_t V, const int64_t *scene_offsets, int32_t n_scenes,
                          int64_t instances, sdgr_caps *out);

/* Device bytes a workspace of these capacities needs (host only).  Returns
 * SDGR_ERR_INVALID for negative or overflowing capacities. */
sdgr_status sdgr_workspace_size(const sdgr_cfg *cfg, const sdgr_caps *caps, size_t *bytes);

/* Binds a caller-allocated device buffer (256-byte aligned, at least
 * sdgr_workspace_size() bytes) to a new workspace handle.  The buffer must
 * stay allocated until sdgr_ws_destroy(); one workspace serves one stream at
 * a time.  Queries the current device's attributes (no allocation).
 * Errors: SDGR_ERR_INVALID (NULL, misaligned or too small buffer, bad cfg). */
sdgr_status sdgr_ws_create(sdgr_ws **out, void *device_buffer, size_t bytes, const sdgr_cfg *cfg,
                           const sdgr_caps *caps);
sdgr_status sdgr_ws_destroy(sdgr_ws *ws);

/* Step a1-a5: Mapping and Projection Algorithm (Section II-A-1: eqs. G(x),
 * W, R_r, Sigmaprime, x_r, x_C, x_i).  For every (view, Gaussian of the
 * view's scene): activations, 3D covariance, world->radar transform,
 * computation-plane and imaging-plane centre and conic, imaging
 * normaliser, float32 slant-range depth key, and the 16x16-tile rectangles
 * the K-ellipse touches on each plane.
 * params: device [max_gaussians][12] float32 (layout above); it must stay
 *   unchanged until sdgr_render_bwd() of this step has run.
 * scene_offsets: host [n_scenes + 1]; views: host [V].
 * Errors: SDGR_ERR_INVALID on bad views / scenes / capacities exceeded. */
sdgr_status sdgr_preprocess(sdgr_ws *ws, const float *params, const int64_t *scene_offsets, int32_t n_scenes,
                            const sdgr_view *views, int32_t V, void *stream);

/* Step a6: bins and sorts.  Per view, a stable radix sort of the depth keys
 * (ties by Gaussian index, the depth-indexed lists of Section II-A); then
 * the (plane, view, tile) instances are emitted in depth order and radix
 * sorted by tile, which keeps depth order within each computation-plane
 * tile; per-tile [start, end) ranges.  If the instances exceed
 * max_instances the status word gets SDGR_ERR_CAPACITY and the required
 * count, and the later kernels of the step skip their work.
 * Errors: SDGR_ERR_STATE if sdgr_preprocess() has not run. */
sdgr_status sdgr_bin_sort(sdgr_ws *ws, void *stream);

/* Steps a7-a8: the scattering-intensity pass on the computation plane
 * (Section II-A-2, eq. I_i: rays from the cell centres, front-to-back
 * compositing with two-way attenuation) and the imaging splat on the
 * range-azimuth plane (Section II-A-3, eq. S_{n,m}: the layover sum).
 * images: device, sum over views of NR*NA float32, overwritten.
 * intensity: device [max_view_gauss] float32 or NULL; if given, receives
 *   I_i per (view, Gaussian) in view order (view v's block starts at the sum
 *   of the earlier views' scene sizes).
 * Errors: SDGR_ERR_STATE if sdgr_bin_sort() has not run. */
sdgr_status sdgr_render_fwd(sdgr_ws *ws, float *images, float *intensity, void *stream);

/* Steps a10-a12: adjoint of the imaging splat (Section II-B-1), of the
 * intensity pass (Section II-B-2; per-ray transmittance is recomputed back
 * to front, not stored per pair) and of the projections (Section II-B-3),
 * summed over the views of each scene.
 * dL_dimages: device, laid out like `images`.
 * grads: device [max_gaussians][12] float32, 16-byte aligned.  accumulate =
 *   0: overwritten for every Gaussian of every scene listed in the last
 *   sdgr_preprocess() call (zero for scenes without views); accumulate = 1:
 *   the gradient is added to what grads holds (e.g. views rendered in
 *   separate calls).
 * Errors: SDGR_ERR_STATE if sdgr_render_fwd() has not run on this workspace
 * since the last sdgr_preprocess(). */
sdgr_status sdgr_render_bwd(sdgr_ws *ws, const float *dL_dimages, float *grads, int32_t accumulate, void *stream);

/* View-dependent scattering (the phase function "from the centre and the
 * spherical harmonic coefficients" of Section II-B-3; SH degree schedule of
 * Section III-B-3).  With plane-wave geometry the direction is the same for
 * every Gaussian of a view: the unit vector d toward the radar,
 * d = (cos theta cos phi, -cos theta sin phi, sin theta).  Then
 *   P_i(view) = P_i + sum_{l=1..degree} sum_m sh_i[l^2 - 1 + l + m] Y_lm(d)
 * with the real orthonormal spherical harmonics (no Condon-Shortley phase),
 * ordered per degree as l=1: (y, z, x); l=2: xy, yz, 3z^2-1, xz, x^2-y^2;
 * l=3: y(3x^2-y^2), xyz, y(5z^2-1), z(5z^2-3), x(5z^2-1), z(x^2-y^2),
 * x(x^2-3y^2) (each times its normalising constant); P_i (parameter 7) is
 * the degree-0 term.
 * sh: device [max_gaussians][16] float32 (entries 15 unused), read by the
 *   following sdgr_preprocess / sdgr_render_bwd calls; NULL disables.
 * dsh: device [max_gaussians][16] float32 or NULL; if given, sdgr_render_bwd
 *   writes dL/dsh there (overwritten or accumulated like grads).
 * degree: 0..3.  Errors: SDGR_ERR_INVALID (degree out of range, NULL ws,
 *   misaligned pointers). */
sdgr_status sdgr_set_sh(sdgr_ws *ws, const float *sh, float *dsh, int32_t degree);

/* Raster schedule (no counterpart in the paper: a launch policy of this
 * library; results do not depend on it beyond float32 atomic order).
 * Every sdgr_bin_sort also builds, per plane, a work list of the tiles whose
 * instance list is non-empty, longest list first (bucketed by the bit length
 * of the list size).  mode:
 *   0: one CTA per tile of the plane, in tile order (every tile launched);
 *   SDGR_SCHED_ORDERED: one CTA per work-list item (empty tiles cost no
 *     work; the images are zeroed before the splat);
 *   SDGR_SCHED_ORDERED | SDGR_SCHED_PERSISTENT: SMs x (CTAs per SM) resident
 *     CTAs pull work-list items from a device counter until the list is
 *     exhausted (no waits between CTAs).
 * Read by the following sdgr_render_fwd / sdgr_render_bwd calls.  Default:
 * SDGR_SCHED_ORDERED | SDGR_SCHED_PERSISTENT.  Errors: SDGR_ERR_INVALID (NULL ws, unknown bits,
 * PERSISTENT without ORDERED). */
#define SDGR_SCHED_ORDERED 1
#define SDGR_SCHED_PERSISTENT 2
sdgr_status sdgr_set_schedule(sdgr_ws *ws, int32_t mode);

/* Staging batch of raster kernel `kernel` (0 intensity pass, 1 splat,
 * 2 splat adjoint, 3 intensity adjoint): the number of Gaussian records a
 * CTA stages into shared memory before its warps walk them (the tile's
 * depth-ordered list is processed in such batches, one barrier pair each).
 * Larger batches mean fewer barriers and less waiting for the slowest warp of
 * a batch; smaller ones less shared memory per CTA (more resident CTAs) and
 * less staging past the point where every ray of a tile has stopped.
 * The result does not depend on it: every pair's arithmetic, the order of
 * each pixel's and ray's sums and every per-(tile, Gaussian) partial sum are
 * the same for every size (the order of the float atomics that add those
 * partial sums across tiles is unordered in any case).
 * sdgr_stage_batch_options writes up to max_sizes supported sizes of
 * `kernel` to sizes (the first is the default) and returns how many there are
 * (0 for an unknown kernel).  sdgr_set_stage_batch selects one of them for
 * the following sdgr_render_fwd / sdgr_render_bwd calls on ws; records = 0
 * restores the default.  Errors: SDGR_ERR_INVALID (NULL ws, unknown kernel,
 * unsupported size). */
int32_t sdgr_stage_batch_options(int32_t kernel, int32_t *sizes, int32_t max_sizes);

/* Device self-check of the approximate instructions whose exact values the
 * kernels rely on.  Writes (asynchronously, on `stream`) a bit mask to the
 * caller's device word *flags: bit 0 set when rcp.approx(1.0f) is exactly
 * 1.0f (the intensity adjoint divides the transmittance by 1 - alpha = 1 for
 * the pairs outside the cutoff, and must leave its bits unchanged).  Every
 * defined bit is set on a correct device (SDGR_SELFCHECK_ALL).  Errors:
 * SDGR_ERR_INVALID (NULL or misaligned flags), SDGR_ERR_CUDA (launch). */
#define SDGR_SELFCHECK_ALL 1u
sdgr_status sdgr_device_selfcheck(uint32_t *flags, void *stream);

/* Diagnostic: the sustained per-SM rate of the instruction kinds the raster
 * kernels are built from, measured on the current device -- the
 * denominators of their arithmetic roofline.  Writes
 * rates[0 .. SDGR_PIPE_RATE_KINDS - 1], each in thread-instructions per SM per
 * SM clock cycle (read from the SM's cycle counter, so independent of the
 * clock frequency): [0] fma.rn.f32, [1] ex2.approx.ftz.f32,
 * [2] rcp.approx.ftz.f32 (each followed by a dependent fma, which is not
 * counted), [3] a stream of one ex2 per seven fma and [4] one rcp per eight
 * fma (all instructions counted; 8 rates[0] / rates[3] - 7 and
 * 9 rates[0] / rates[4] - 8 are what one ex2 and one rcp cost inside an FP32
 * stream, in fma issue slots), [5] fma.rn.f32x2 (two FMAs each),
 * [6] fma.rn.f32 and lop3.b32 alternating, [7] fma.rn.f32x2 and lop3.b32
 * alternating (all instructions counted).
 * scratch: caller-owned device memory of at least SDGR_PIPE_RATES_SCRATCH
 * bytes, 16-byte aligned.  Synchronous (waits for `stream`; a few ms).
 * Errors: SDGR_ERR_INVALID (NULL or misaligned arguments), SDGR_ERR_CUDA. */
#define SDGR_PIPE_RATES_SCRATCH 8192
#define SDGR_PIPE_RATE_KINDS 8
sdgr_status sdgr_pipe_rates(void *scratch, double *rates, void *stream);
sdgr_status sdgr_set_stage_batch(sdgr_ws *ws, int32_t kernel, int32_t records);

/* Densification and pruning (the "Densification and Pruning Operation" of
 * Section II-B and the thresholds of Section III-D).  Gradient statistics:
 * while bound, every sdgr_render_bwd adds, for each Gaussian and each view
 * in which it received any image-plane weight, the norm of its image-plane
 * positional gradient |dL/du_I| (pixel units) to accum[i] and 1 to
 * count[i] (device float32 [max_gaussians]; the caller zeroes them at the
 * start of an accumulation window).  NULL pointers unbind. */
sdgr_status sdgr_set_densify_stats(sdgr_ws *ws, float *accum, float *count);

/* Densification rules (all comparisons in float32):
 * grad_threshold  densify Gaussians with count > 0 and accum/count > it
 *                 (default 0.003)
 * dense_scale     densified Gaussians whose largest scale is <= it are
 *                 cloned (the copy moved by its largest scale along
 *                 -dL/dmu), larger ones are split in two (children half
 *                 their largest scale from the centre along that axis,
 *                 child 0 on the -dL/dmu side, log-scales - ln split_factor)
 * max_scale       prune if the largest scale exceeds it (0.3 x the
 *                 illuminated extent)
 * min_opacity     prune if sigmoid(opacity logit) < it
 * min_P           prune if P < it (backscattering too small)
 * split_factor    scale divisor of split children (1.6) */
typedef struct {
    float grad_threshold;
    float dense_scale;
    float max_scale;
    float min_opacity;
    float min_P;
    float split_factor;
} sdgr_densify_cfg;

/* Bytes of device scratch sdgr_densify needs for N Gaussians (host only). */
size_t sdgr_densify_scratch_bytes(int64_t N);

/* Applies the rules to N Gaussians.  In: params, grads (dL/dparams of the
 * last step; its mean part sets the displacement direction), accum, count
 * (device, as above), m, v (Adam moments, device [N][12]), sh (device
 * [N][16] or NULL).  Out: out_params, out_m, out_v (device [out_capacity][12])
 * and out_sh (device [out_capacity][16], iff sh): Gaussian i's survivors
 * appear in order -- kept (its moments carried over), kept + clone, or the
 * two split children -- new Gaussians with zero moments.  scratch: device,
 * sdgr_densify_scratch_bytes(N) bytes.  *new_N (host) receives the output
 * count.  Synchronous: waits for `stream` to read the count.
 * Errors: SDGR_ERR_INVALID; SDGR_ERR_CAPACITY if the output would exceed
 * out_capacity (*new_N then holds the required count, nothing is written). */
sdgr_status sdgr_densify(const float *params, const float *grads, const float *accum, const float *count,
                         const float *m, const float *v, const float *sh, int64_t N, const sdgr_densify_cfg *cfg,
                         float *out_params, float *out_m, float *out_v, float *out_sh, int64_t out_capacity,
                         void *scratch, int64_t *new_N, void *stream);

/* Step a13: the optimiser step of the training loop (Section II: the
 * Gaussians' parameters are updated by gradient descent on the loss; the
 * paper names no optimiser, so the update is read as Adam -- Kingma & Ba,
 * bias-corrected, eps added to the square root of the corrected second
 * moment, torch.optim.Adam semantics, no weight decay -- as in the 3D
 * Gaussian splatting training the paper builds on).  Over N Gaussians.  params, grads, m, v: device
 * [N][12] float32, 16-byte aligned; params, m, v updated in place.  lr: host
 * [5] learning rates for the groups {means, log-scales, quaternions,
 * opacity logit, P}.  step: 1-based step count.
 * Errors: SDGR_ERR_INVALID (N < 0, step < 1, misaligned pointers). */
sdgr_status sdgr_adam_step(float *params, const float *grads, float *m, float *v, int64_t N, const float *lr,
                           float b1, float b2, float eps, int32_t step, void *stream);

/* Step a13 for any other trained float32 array (the SH coefficients of the
 * view-dependent scattering): the same Adam update with one learning rate
 * for every element.  x, grads, m, v: device [n] float32, 16-byte aligned,
 * n a multiple of 4; x, m, v updated in place.
 * Errors: SDGR_ERR_INVALID (n < 0 or not a multiple of 4, step < 1,
 * misaligned pointers). */
sdgr_status sdgr_adam_step_flat(float *x, const float *grads, float *m, float *v, int64_t n, float lr, float b1,
                                float b2, float eps, int32_t step, void *stream);

/* Step a13, graph-replayable form: as sdgr_adam_step, but the 1-based step
 * count lives in device memory.  step: device int32; the call increments
 * *step first and uses the new value, so a captured CUDA graph that
 * contains this call applies the right bias correction at every replay.
 * Errors: SDGR_ERR_INVALID (N < 0, NULL step, misaligned pointers). */
sdgr_status sdgr_adam_step_device(float *params, const float *grads, float *m, float *v, int64_t N, const float *lr,
                                  float b1, float b2, float eps, int32_t *step, void *stream);

/* Step a9: L1 loss, mean over npix pixels, and dL/dS = sign(S - S*)/npix
 * (sign(0) = 0).  images, targets, dL_dimages: device [npix] float32; loss:
 * device float32 scalar, overwritten.  Errors: SDGR_ERR_INVALID. */
sdgr_status sdgr_l1_loss(const float *images, const float *targets, int64_t npix, float *dL_dimages, float *loss,
                         void *stream);

/* Reads the workspace's device status word (a synchronous device-to-host
 * copy: call after the stream has finished).  Returns SDGR_OK or the device
 * status (SDGR_ERR_CAPACITY / SDGR_ERR_TIMEOUT); *required_instances (may be
 * NULL) receives the instance count the last sdgr_bin_sort() needed. */
sdgr_status sdgr_read_status(sdgr_ws *ws, int64_t *required_instances);

/* Stage timing.  With profiling enabled, the workspace brackets each
 * kernel stage of sdgr_preprocess / sdgr_bin_sort / sdgr_render_fwd /
 * sdgr_render_bwd with CUDA events recorded on the launching stream (the
 * events are created by sdgr_profile_enable; no device memory is
 * allocated).  sdgr_profile_read waits for the recorded events, and adds
 * up, per stage, the elapsed milliseconds and the number of launches since
 * the last reset.  ms and launches: host arrays of SDGR_NUM_STAGES entries.
 * Calls enqueued on a stream that is being captured into a CUDA graph record
 * their events as event-record nodes of the graph: every replay records
 * them again, and sdgr_profile_read, called after a replay has finished,
 * adds that replay's stage times (read once: the read resets the record of
 * which events are pending).
 * Errors: SDGR_ERR_INVALID (NULL ws / arrays), SDGR_ERR_CUDA. */
enum {
    SDGR_STAGE_PREPROCESS = 0,   /* step a1-a5 */
    SDGR_STAGE_DEPTH_SORT = 1,   /* step a6: per-view depth radix sort */
    SDGR_STAGE_BIN = 2,          /* step a6: counts, emission, tile sort, ranges */
    SDGR_STAGE_INTENSITY_FWD = 3,/* step a7 */
    SDGR_STAGE_SPLAT_FWD = 4,    /* step a8 */
    SDGR_STAGE_SPLAT_BWD = 5,    /* step a10 */
    SDGR_STAGE_INTENSITY_BWD = 6,/* step a11 */
    SDGR_STAGE_PARAM_BWD = 7,    /* step a12 */
    SDGR_NUM_STAGES = 8
};
sdgr_status sdgr_profile_enable(sdgr_ws *ws, int32_t enable);
sdgr_status sdgr_profile_read(sdgr_ws *ws, double *ms, int64_t *launches, int32_t reset);

/* Diagnostics.  sdgr_count_pairs counts, for the current sorted lists, the
 * (pixel, Gaussian) pairs inside the cutoff ellipse on the computation plane
 * (pairs[0]) and on the imaging plane (pairs[1]); it is synchronous (waits
 * for `stream`).  sdgr_launch_count returns the number of kernels the
 * library has launched in this process. */
sdgr_status sdgr_count_pairs(sdgr_ws *ws, int64_t *pairs, void *stream);
int64_t sdgr_launch_count(void);

/* Forward render without any device allocation, for callers that cannot
 * allocate device memory: code running where cudaMalloc is not available to
 * it (a plugin inside a host application that owns all device memory
 * through its own allocator, a real-time loop that must not allocate after
 * start-up) still has to render small scenes.  The paper has no counterpart;
 * this is a library convenience.
 *
 * Same computation and outputs as sdgr_preprocess + sdgr_bin_sort +
 * sdgr_render_fwd on one scene, but the workspace is a fixed
 * SDGR_NOALLOC_SCRATCH_BYTES (32 MiB) array in the library's own device
 * memory, reserved once on every GPU that loads the library and kept until
 * the process exits.  Limits: N <= SDGR_NOALLOC_MAX_GAUSSIANS, 1 <= V <=
 * SDGR_NOALLOC_MAX_VIEWS, sum of NA*NR <= SDGR_NOALLOC_MAX_PIXELS, every
 * view's scene == 0; larger requests return SDGR_ERR_INVALID, and a scene
 * whose tile instances do not fit the scratch returns SDGR_ERR_CAPACITY
 * (images then hold zeros).
 * params: device [N][12] float32 (16-byte aligned); views: host [V];
 * images: device, sum of NA*NR float32, overwritten; intensity: device [V*N]
 * float32 or NULL.
 * The first call on a device looks up the scratch array's device address
 * (once per device, with that device current), so make that first call
 * before any stream capture.  The call waits for `stream` before it returns
 * (it reads the device status word).  Every call reuses the
 * same scratch, which keeps the previous call's contents (everything that
 * must start at zero is cleared by the call); host threads are serialised by
 * a lock, but calls whose work overlaps on the GPU (e.g. from two processes
 * sharing the device) race on the scratch. */
#define SDGR_NOALLOC_SCRATCH_BYTES (32u << 20)
#define SDGR_NOALLOC_MAX_GAUSSIANS 16384
#define SDGR_NOALLOC_MAX_VIEWS 4
#define SDGR_NOALLOC_MAX_PIXELS 262144
sdgr_status sdgr_render_fwd_noalloc(const float *params, int64_t N, const sdgr_view *views, int32_t V,
                                    const sdgr_cfg *cfg, float *images, float *intensity, void *stream);

/* Asynchronous form of sdgr_read_status: enqueues on `stream` a copy of the
 * status word into `host_dst` (caller-owned page-locked host memory of at
 * least 16 bytes): int32 status code, int32 reserved, int64 instances the
 * last sdgr_bin_sort needed.  Valid once the stream has reached that point
 * (e.g. after an event recorded behind it has completed).
 * Errors: SDGR_ERR_INVALID (NULL arguments), SDGR_ERR_CUDA. */
sdgr_status sdgr_copy_status_async(sdgr_ws *ws, void *host_dst, void *stream);

/* Static, NUL-terminated description of a status code. */
const char *sdgr_status_string(sdgr_status s);

#ifdef __cplusplus
}
#endif

#endif /* SDGR_H */
