/*
 * pa.h -- C ABI of the GB300 (sm_103a) library for the data-parallel hot path
 * of 4D SlingBAG (arXiv 2412.03898): per-frame Gaussian-basis deformation of
 * a Gaussian-ball point cloud, photoacoustic forward projection of every ball
 * into every sensor trace, the L2 data-fidelity loss, and the adjoint back to
 * ball and deformation parameters.
 *
 * Conventions (all entry points)
 * ------------------------------
 *  - Units: lengths in mm, times in microseconds, sampling rate in MHz,
 *    sound speed in mm/us.
 *  - A ball state has five channels in this order: x, y, z (centre mu),
 *    a (Gaussian standard deviation, "size" a0) and p (peak initial pressure
 *    p0) -- the attributes of Sec. 2.1.  Ball arrays are structure-of-arrays
 *    with a channel stride `stride` (elements), stride >= n and
 *    stride % 4 == 0, and base pointers 16-byte aligned; elements between n
 *    and stride are never used but must be readable (the library copies whole
 *    16-byte granules).
 *  - Pointers named "device" are CUDA device pointers; "host" pointers are
 *    host memory.  The caller owns every buffer; the library allocates no
 *    device memory.  Scratch memory is a caller-provided workspace whose size
 *    is returned by the matching *_workspace_size query.
 *  - Every call is asynchronous on the caller's stream (`stream` is a
 *    cudaStream_t; NULL = legacy default stream) and returns a status code.
 *    Argument errors are detected on the host before anything is launched
 *    (PA_ERR_INVALID_ARG).  Data-dependent errors found inside kernels (a
 *    sensor inside a ball's support, a non-positive basis width, a bounded
 *    wait that ran out) are recorded in a per-device error word and read back
 *    by pa_device_error().
 *  - Outputs are overwritten unless PA_ACCUMULATE is set in `flags`, in which
 *    case results are added to the existing contents.
 *
 * The radiator.  The paper drives its reconstruction with SlingBAG's
 * differentiable forward model (Sec. 2.2, last paragraph) without printing
 * its formula.  This library uses the exact solution of the 3D wave equation
 * for a Gaussian initial pressure p*exp(-|x-mu|^2/(2a^2)) with zero initial
 * velocity.  At a sensor at distance R from mu, sampled at t_k = t0 + k/fs,
 *     y[k] += p/(2R) * tau * exp(-tau^2/(2a^2)),   tau = R - c t_k,
 * on the closed window |tau| <= kappa*a (the "arrival window" of the ball),
 * the inward-travelling term being below (R/a) exp(-R^2/(2a^2)) of the peak.
 */
#ifndef PA_H
#define PA_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__) || defined(__clang__)
#define PA_API __attribute__((visibility("default")))
#else
#define PA_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes. */
#define PA_OK 0
#define PA_ERR_INVALID_ARG 1 /* bad pointer, size, alignment or scalar */
#define PA_ERR_DOMAIN 2      /* sensor inside a ball's support (R <= kappa a), or sigma_n <= 0 */
#define PA_ERR_CUDA 3        /* a CUDA runtime call failed (launch, attribute, copy) */
#define PA_ERR_TIMEOUT 4     /* a bounded wait inside a kernel ran out */
#define PA_ERR_WORKSPACE 5   /* workspace NULL, misaligned or smaller than required */

/* Flags. */
#define PA_ACCUMULATE 1u      /* add into the output instead of overwriting it */
#define PA_SSIM_MINMAX 4u     /* pa_ssim only: scale each image to [0, 1] by its own minimum and
                                 maximum first (a constant image becomes 0), L = 1 */
#define PA_PROFILE_UNIFORM 2u /* pa_forward only: uniform ball of radius a (N-pulse
                                 p tau/(2R) on |tau| <= a), used for analytic tests */
#define PA_PLAN_TUNE 8u       /* pa_plan_create only: time candidate plans on the caller's data */

/* Scratch bytes of pa_adjoint's optional work-queue workspace. */
#define PA_ADJOINT_WORKSPACE_BYTES 256u

/* Acquisition geometry.  `sensors` is a device array [3][sensor_stride]
 * (x row, y row, z row) of sensor positions.  Constraints: n_sensors >= 1,
 * sensor_stride >= n_sensors, c > 0, fs > 0, t0 >= 0, n_samples >= 4 and a
 * multiple of 4, 1 <= kappa <= 8.  The paper's arrays are sparse 2D arrays
 * on spheres with Fibonacci layouts (Sec. 3.1, Sec. 3.2). */
typedef struct pa_geom {
    const float *sensors;
    int32_t n_sensors;
    int32_t sensor_stride;
    float c;         /* speed of sound, mm/us */
    float fs;        /* sampling rate, MHz */
    float t0;        /* time of sample 0, us */
    int32_t n_samples; /* T */
    float kappa;     /* window half-width in units of a */
} pa_geom;

/* Per-frame ball states (Eq. 1 outputs, or a static SlingBAG cloud):
 * device array [n_frames][5][stride], channels x, y, z, a, p. */
typedef struct pa_balls {
    const float *state;
    int64_t n;
    int64_t stride;
} pa_balls;

/* GGBall parameters (Sec. 2.2, Eq. 1-2): canonical cloud `canon`
 * [5][stride] and, per channel, ball and basis function, the weight omega,
 * centre theta and width sigma of the Gaussian basis, each device
 * [5][n_basis][stride].  1 <= n_basis <= 128 (the paper uses 65). */
typedef struct pa_canon {
    const float *canon;
    const float *omega;
    const float *theta;
    const float *sigma;
    int64_t n;
    int64_t stride;
    int32_t n_basis;
} pa_canon;

/* Gradient outputs of pa_adjoint.  Static mode: `state` is
 * [n_frames][5][stride] = dL/d(per-frame state); omega/theta/sigma unused.
 * 4D mode: `state` is [5][stride] = dL/d(canonical cloud) and
 * omega/theta/sigma are [5][n_basis][stride]. */
typedef struct pa_grads {
    float *state;
    float *omega;
    float *theta;
    float *sigma;
} pa_grads;

/* One scene of a batched call: its own sensor array, acquisition scalars,
 * per-frame ball states and outputs.  Scenes may differ in every size. */
typedef struct pa_scene {
    pa_geom geom;
    pa_balls balls;          /* device [n_frames][5][stride] */
    int32_t n_frames;
    float *traces;           /* pa_forward_batched output, device [n_frames][S][T], 16-byte aligned */
    const float *trace_grad; /* pa_adjoint_batched input, device [n_frames][S][T], 16-byte aligned */
    float *grad_state;       /* pa_adjoint_batched output, device [n_frames][5][stride] */
} pa_scene;

/* Most scenes one batched call takes. */
#define PA_MAX_SCENES 64

/* Launch plan (opaque, host memory): the forward's tiles (sensors and samples
 * per CTA, balls per TMA stage, ball splits, pairs swept together), the frames
 * per launch of the 4D calls, and the (scene, frame, ball) items per queue
 * grab of the batched adjoint.  Made by pa_plan_create (heuristic or timed on
 * the caller's data) or pa_plan_from_values, released by pa_plan_destroy.
 * A plan is read-only during the calls that take it; NULL means the built-in
 * heuristic everywhere. */
typedef struct pa_plan pa_plan;

/* A voxel grid [nz][ny][nx] (x fastest); voxel (ix, iy, iz) is centred at
 * origin + h (ix, iy, iz), in mm.  h > 0; nx, ny, nz >= 1. */
typedef struct pa_grid {
    float origin[3];
    float h;
    int32_t nx, ny, nz;
} pa_grid;

/* Human-readable name of a status code (static storage). */
PA_API const char *pa_status_string(int32_t status);

/* Library ABI version (major*100 + minor).  1.01 added pa_deform_backward,
 * the imaging calls (pa_ubp_filter, pa_ubp, pa_splat, pa_map, pa_ssim*) and
 * pa_selftest_bounded_wait.  2.00 added launch plans (pa_plan_*), the 4D
 * calls that recompute states per frame chunk (pa_forward_4d,
 * pa_adjoint_4d) and pa_measure_unit_rates, changed pa_forward_batched and
 * pa_adjoint_batched to take a plan in place of a tile array, and
 * pa_batched_workspace_size to take the scenes and the plan.  2.01 gave
 * pa_adjoint an optional work-queue workspace; 2.02 added pa_spatial_order
 * and pa_gather_rows. */
PA_API int32_t pa_version(void);

/* Reads, returns in *out (host) and clears the device error word of the
 * current device.  Synchronises `stream`.  *out is PA_OK or the first
 * data-dependent error recorded by a kernel since the last call. */
PA_API int32_t pa_device_error(void *stream, int32_t *out);

/* Eq. 1-2 (Sec. 2.2): deformed state of every ball at every frame,
 *   q(t_f) = q0 (1 + sum_n omega_n exp(-(t_f - theta_n)^2 / (2 sigma_n^2)))
 * for q in (x, y, z, a, p), one independent H per channel.
 *   t_frames  device [n_frames] normalised frame times (t_f = f/(F-1) in the
 *             paper's reading of "normalized time frame")
 *   state_out device [n_frames][5][canon->stride]
 * sigma_n <= 0 records PA_ERR_DOMAIN (that term is skipped). */
PA_API int32_t pa_deform_balls(const pa_canon *canon, const float *t_frames, int32_t n_frames,
                        float *state_out, void *stream);

/* Chain rule of Eq. 1-2 (Sec. 2.2; the paper makes every (theta, sigma,
 * omega) and the canonical attributes learnable) on its own: from per-frame
 * state gradients
 *   g_state   device [n_frames][5][canon->stride] = dL/d(state at t_f), e.g.
 *             the static-mode pa_adjoint output for the states that
 *             pa_deform_balls produced for the same t_frames,
 * writes dL/d(canonical cloud) to grads->state [5][stride] and
 * dL/d(omega, theta, sigma) to grads->omega / theta / sigma
 * [5][n_basis][stride] (all device, caller-owned).  pa_deform_balls, the
 * static pa_adjoint and this call give pa_adjoint's 4D mode up to float
 * summation order, at the cost of two [n_frames][5][stride] buffers; the
 * static adjoint runs at higher occupancy than the fused 4D kernel.
 * flags: PA_ACCUMULATE adds to the outputs.  sigma_n <= 0 records
 * PA_ERR_DOMAIN and that term gets zero gradient. */
PA_API int32_t pa_deform_backward(const pa_canon *canon, const float *t_frames, int32_t n_frames,
                                  const float *g_state, pa_grads *grads, uint32_t flags, void *stream);

/* Scratch bytes pa_forward needs for this problem (0 if none). */
PA_API size_t pa_forward_workspace_size(const pa_geom *geom, const pa_balls *balls, int32_t n_frames);

/* Forward projection (Sec. 2.2, last paragraph; Sec. 2.1): for every frame f,
 * sensor s and sample k, the sum over balls of the radiated pulse above.
 *   traces    device [n_frames][n_sensors][n_samples], 16-byte aligned
 *   workspace device scratch of at least pa_forward_workspace_size() bytes,
 *             256-byte aligned (may be NULL when the size is 0)
 * Balls with a <= 0 or p == 0 contribute nothing; a pair with R <= kappa a is
 * skipped and records PA_ERR_DOMAIN.  Deterministic: the same inputs give
 * bitwise the same traces. */
PA_API int32_t pa_forward(const pa_geom *geom, const pa_balls *balls, int32_t n_frames, float *traces,
                   uint32_t flags, void *workspace, size_t workspace_bytes, void *stream);

/* pa_forward with an explicit tile plan, for autotuning.  tiles = {sensors
 * per CTA (1..16, 0 = default), samples per CTA (multiple of 4, 0 = default),
 * balls per TMA stage (multiple of 4, at most 8192, 0 = default), ball splits (0 =
 * default), pairs swept together per warp (1, 2, 4, 8 or 16; 0 = default)}, a
 * host array of 5, or NULL for the built-in heuristic.  Results equal
 * pa_forward's up to float summation order. */
PA_API size_t pa_forward_workspace_size_ex(const pa_geom *geom, const pa_balls *balls, int32_t n_frames,
                                           const int32_t *tiles);
PA_API int32_t pa_forward_ex(const pa_geom *geom, const pa_balls *balls, int32_t n_frames, float *traces,
                             uint32_t flags, const int32_t *tiles, void *workspace, size_t workspace_bytes,
                             void *stream);

/* The plan pa_forward_ex would use: out7 (host) receives {sensors per CTA,
 * samples per CTA, balls per stage, ball splits, pairs per sweep, CTAs
 * launched, dynamic shared memory bytes per CTA}. */
PA_API int32_t pa_forward_plan_info(const pa_geom *geom, const pa_balls *balls, int32_t n_frames,
                                    const int32_t *tiles, int32_t *out7);

/* Adjoint of pa_forward (gradients of the L2 loss, Sec. 2.2, last paragraph:
 * all baseline attributes and all (theta, sigma, omega) are learnable).
 * Given trace_grad = dL/dy, device [n_frames][n_sensors][n_samples] (16-byte
 * aligned, read as float pairs), and an
 * optional per-frame scale (device [n_frames] or NULL = 1) applied to it:
 *  - static mode (balls != NULL, canon == NULL): grads->state receives
 *    dL/d(x, y, z, a, p) per frame;
 *  - 4D mode (balls == NULL, canon != NULL, t_frames device [n_frames]):
 *    the per-frame state is recomputed from Eq. 1-2 inside the kernel (never
 *    stored) and the chain rule of Eq. 1-2 gives dL/d(canonical cloud) and
 *    dL/d(omega, theta, sigma), summed over frames.
 * Every per-ball gradient is written by exactly one warp: no atomics, and
 * deterministic.  Inactive balls (a <= 0 or p == 0) get zero state gradient.
 * workspace: NULL, or device scratch of at least PA_ADJOINT_WORKSPACE_BYTES
 * aligned to 256 bytes (else PA_ERR_WORKSPACE), which static mode uses as a
 * work-queue counter: persistent warps then take (frame, ball) items from
 * it, so warps that drew small windows take more items.  With NULL the items
 * are dealt out in a fixed grid-stride order.  The results are identical
 * either way (each item is computed whole by one warp); 4D mode ignores the
 * workspace.  One workspace serves one call at a time: calls in flight on
 * different streams need their own. */
PA_API int32_t pa_adjoint(const pa_geom *geom, const pa_balls *balls, const pa_canon *canon,
                   const float *t_frames, int32_t n_frames, const float *trace_grad,
                   const float *frame_scale, pa_grads *grads, uint32_t flags, void *workspace,
                   size_t workspace_bytes, void *stream);

/* Scratch bytes the batched calls need for these scenes and this plan
 * (NULL: the heuristic): the work-queue counter (256 bytes, all that
 * pa_adjoint_batched uses) and, for pa_forward_batched, the partial traces
 * [splits][F][S][T] of every scene it splits by balls. */
PA_API size_t pa_batched_workspace_size(const pa_scene *scenes, int32_t n_scenes, const pa_plan *plan);

/* Forward projection of several independent scenes of uneven ball, sensor,
 * sample and frame counts in one persistent launch (the batching of Sec. 1:
 * one cloud per scene for all its frames; several scenes per launch).  The
 * work items (scene, frame, sensor tile, sample tile, ball split) are taken
 * from a counter in the workspace, scenes with the most balls per split
 * first, by one CTA per SM.  A scene is split into ball ranges (the plan's
 * split count, else one per 131072 balls), whose partial traces are summed
 * in split order afterwards with compensated additions; with one split its
 * traces equal pa_forward_ex's with the same tiles and one split.
 * scenes: host array of n_scenes (<= PA_MAX_SCENES); plan: tiles and split
 * count, or NULL for the heuristic; workspace: device, 256-byte aligned, at
 * least pa_batched_workspace_size(scenes, n_scenes, plan) bytes.  Only the
 * Gaussian profile; flags: PA_ACCUMULATE. */
PA_API int32_t pa_forward_batched(const pa_scene *scenes, int32_t n_scenes, uint32_t flags, const pa_plan *plan,
                                  void *workspace, size_t workspace_bytes, void *stream);

/* Static-mode adjoint of several scenes in one persistent launch: warps take
 * chunks of (scene, frame, ball) items from a counter in the workspace,
 * scenes with the most sensors first; plan: its items per grab, or NULL
 * (1).  Each scene's grad_state equals pa_adjoint's static mode.  flags:
 * PA_ACCUMULATE. */
PA_API int32_t pa_adjoint_batched(const pa_scene *scenes, int32_t n_scenes, uint32_t flags, const pa_plan *plan,
                                  void *workspace, size_t workspace_bytes, void *stream);

/* Device workspace bytes pa_plan_create needs to time candidates on these
 * scenes (the largest forward workspace among the candidate tiles of a
 * single scene, or a batched call's queue counter). */
PA_API size_t pa_plan_workspace_size(const pa_scene *scenes, int32_t n_scenes);

/* Launch plan for scenes like these (Sec. 1 and Sec. 2.2 batching; the
 * paper prints no launch configuration, so the tiles come from this tuner).
 * Without PA_PLAN_TUNE the plan holds the built-in heuristic and nothing is
 * launched.  With PA_PLAN_TUNE the library times every candidate tile plan
 * (best of several CUDA-event-timed runs on `stream`) and keeps the fastest:
 * for one scene through pa_forward_ex (the planner choosing ball splits),
 * for several through pa_forward_batched, and for several scenes that all
 * carry trace_grad and grad_state also the batched adjoint's items per grab.
 * Tuning overwrites the scenes' traces (and grad_state), synchronises
 * `stream` and must not run during stream capture.  workspace: device,
 * 256-byte aligned, at least pa_plan_workspace_size() bytes.  *out receives
 * the plan (host memory owned by the caller until pa_plan_destroy); on an
 * error *out is NULL. */
PA_API int32_t pa_plan_create(const pa_scene *scenes, int32_t n_scenes, uint32_t flags, void *workspace,
                              size_t workspace_bytes, void *stream, pa_plan **out);

/* A plan from explicit values (host int32[7], or NULL for all defaults):
 * {sensors per CTA (1..16), samples per CTA (multiple of 4), balls per stage
 * (multiple of 4, <= 8192), ball splits, pairs per sweep (1, 2, 4, 8, 16),
 * frames per 4D launch, batched-adjoint items per grab (<= 1024)}, 0 = the
 * heuristic for that entry.  For tuned values from another process or a
 * cache. */
PA_API int32_t pa_plan_from_values(const int32_t *values7, pa_plan **out);

/* Reads a plan: values7 (host int32[7], same order as pa_plan_from_values)
 * and, if timings2 != NULL, the best forward and batched-adjoint times in ms
 * measured while tuning (0 when not tuned). */
PA_API int32_t pa_plan_get(const pa_plan *plan, int32_t *values7, float *timings2);

/* Releases a plan (NULL is ignored). */
PA_API void pa_plan_destroy(pa_plan *plan);

/* Scratch bytes pa_forward_4d needs: one frame chunk of deformed states
 * [K][5][stride] plus the forward's split partials for K frames. */
PA_API size_t pa_forward_4d_workspace_size(const pa_geom *geom, const pa_canon *canon, int32_t n_frames,
                                           const pa_plan *plan);

/* Forward projection of a 4D sequence straight from the GGBall parameters
 * (Eq. 1-2, Sec. 2.2; radiator as pa_forward): frames are processed in
 * chunks of K (the plan's frames per launch, else K = floor(3 n_basis / 16),
 * which keeps a chunk's states and state gradients within an eighth of the
 * deformation parameters' memory), each chunk deformed into the workspace
 * and projected, so the states of at most K frames exist at any time:
 * memory is the canonical cloud, its deformation parameters and one chunk,
 * whatever n_frames is.
 *   t_frames  device [n_frames] normalised frame times
 *   traces    device [n_frames][n_sensors][n_samples], 16-byte aligned
 *   workspace device, 256-byte aligned, pa_forward_4d_workspace_size() bytes
 * flags: PA_ACCUMULATE.  Traces equal pa_deform_balls + pa_forward_ex with
 * the same tiles per chunk. */
PA_API int32_t pa_forward_4d(const pa_geom *geom, const pa_canon *canon, const float *t_frames, int32_t n_frames,
                             float *traces, uint32_t flags, const pa_plan *plan, void *workspace,
                             size_t workspace_bytes, void *stream);

/* Scratch bytes pa_adjoint_4d needs: a work-queue counter (256 bytes) and
 * one frame chunk of states and one of state gradients, [K][5][stride] each. */
PA_API size_t pa_adjoint_4d_workspace_size(const pa_geom *geom, const pa_canon *canon, int32_t n_frames,
                                           const pa_plan *plan);

/* Adjoint of pa_forward_4d (Sec. 2.2: the canonical attributes and every
 * (theta, sigma, omega) are learnable): per frame chunk, the deformed states
 * are recomputed (never stored across chunks), the static adjoint gives their
 * gradients, and the chain rule of Eq. 1-2 adds them into dL/d(canonical
 * cloud) grads->state [5][stride] and dL/d(omega, theta, sigma)
 * [5][n_basis][stride].  trace_grad: device [n_frames][S][T], 16-byte
 * aligned; frame_scale: device [n_frames] or NULL (= 1).  flags:
 * PA_ACCUMULATE.  Equals pa_adjoint's 4D mode up to float summation order,
 * deterministic, no atomics. */
PA_API int32_t pa_adjoint_4d(const pa_geom *geom, const pa_canon *canon, const float *t_frames, int32_t n_frames,
                             const float *trace_grad, const float *frame_scale, pa_grads *grads, uint32_t flags,
                             const pa_plan *plan, void *workspace, size_t workspace_bytes, void *stream);

/* Scratch bytes pa_spatial_order needs for n balls (0 for n <= 0). */
PA_API size_t pa_spatial_order_workspace_size(int64_t n);

/* Spatial (Morton, Z-curve) order of a cloud's ball centres: perm[i] (device
 * int32 [n], caller-owned) is the index of the ball to store at position i.
 * A storage layout aid, not part of the method (every sum of the paper is
 * over all balls, in any order): the forward sweeps tiles of consecutive
 * balls, and a cloud stored in this order gives those tiles tight bounding
 * boxes (on a 100k-ball vessel tree: 5% off the forward of the cloud
 * stored along its tubes, two thirds off that of a randomly ordered one).  Cubic cells of edge h, the power of two nearest to the mean
 * radius a of the balls with a > 0 (at least the largest extent of the
 * centres' bounding box / 1024): cell = floor((x - min_x) / h) clamped to
 * [0, 1023] per axis, the difference one rounded float32 operation; code =
 * interleaved bits (x lowest).  Balls closer than about their own size keep
 * their index order.
 * Equal codes keep their index order: the permutation is deterministic.
 * balls: frame 0 of balls->state is read; n < 2^31.  workspace: device,
 * 256-byte aligned, pa_spatial_order_workspace_size(n) bytes.  Apply it with
 * pa_gather_rows to the state (5 rows) and, for a 4D cloud, to the
 * deformation parameters (5 * n_basis rows each). */
PA_API int32_t pa_spatial_order(const pa_balls *balls, int32_t *perm, void *workspace, size_t workspace_bytes,
                                void *stream);

/* out[r * stride + i] = in[r * stride + perm[i]] for rows r < rows and
 * columns i < n (device arrays; out's padding columns are not written; in and
 * out must not overlap: the same pointer is rejected, other overlaps are not
 * detected).  perm: device int32 [n] with values in [0, n), e.g. from
 * pa_spatial_order (not checked). */
PA_API int32_t pa_gather_rows(const float *in, float *out, int64_t n, int64_t stride, int32_t rows,
                              const int32_t *perm, void *stream);

/* Scratch bytes pa_residual_loss needs. */
PA_API size_t pa_loss_workspace_size(int64_t per_frame, int32_t n_frames);

/* L2 data-fidelity loss (Sec. 2.2, last paragraph), per frame, in FP64:
 *   loss[f]  = sum_i (pred[f][i] - meas[f][i])^2          (device [n_frames], or NULL)
 *   resid[f][i] = 2 scale[f] (pred[f][i] - meas[f][i])     (device, or NULL)
 * pred, meas, resid: device [n_frames][per_frame], 16-byte aligned,
 * per_frame % 4 == 0.  frame_scale: device [n_frames] or NULL (= 1).
 * Deterministic (fixed reduction order). */
PA_API int32_t pa_residual_loss(const float *pred, const float *meas, int64_t per_frame, int32_t n_frames,
                         const float *frame_scale, double *loss, float *resid, void *workspace,
                         size_t workspace_bytes, void *stream);

/* pa_residual_loss without a workspace argument, for callers that cannot
 * allocate device memory where they call it: a plugin whose host application
 * owns every device allocation, or a C caller with no allocator at hand that
 * must not call cudaMalloc (which can implicitly synchronise the device).
 * The paper has no counterpart; this is a deployment variant of the loss.
 * Same arguments, results and determinism as pa_residual_loss.  Its scratch
 * is a fixed 128 KiB array inside the library, held on every GPU that loads
 * the library until the process exits, with room for 16384 (frame, block)
 * partial sums; a frame of P samples takes min(1024, ceil(P / 32768)) blocks,
 * so floor(16384 / blocks) frames fit (for example, 227 frames of 576 x 4096
 * samples, 72 blocks each).  Larger problems
 * return PA_ERR_WORKSPACE without launching anything.  It allocates nothing.
 * The first call on a device looks up that array's device address (with the
 * device current) and caches it per device index for the life of the
 * process; make that first call before any stream capture.  The cached
 * address belongs to the device's primary context: after cudaDeviceReset, or
 * from a different (non-primary) context on the same device, it is stale, so
 * such callers must not use this entry point.  All calls share the one array: calls that overlap on the GPU
 * (two streams or two threads) race and must be serialised by the caller.
 * Each call writes every partial it reads, so the array never needs
 * clearing. */
PA_API int32_t pa_residual_loss_noalloc(const float *pred, const float *meas, int64_t per_frame, int32_t n_frames,
                                        const float *frame_scale, double *loss, float *resid, void *stream);

/* Sum of squares in FP64 of a device float array (gradient norms), written to
 * *out (device double).  n % 4 == 0, x 16-byte aligned. */
PA_API int32_t pa_sumsq(const float *x, int64_t n, double *out, void *workspace, size_t workspace_bytes,
                 void *stream);

/* Number of (frame, sensor, ball, sample) terms pa_forward sums, written to
 * *out (device uint64).  This is the "contribution" count of the throughput
 * metric. */
PA_API int32_t pa_count_contributions(const pa_geom *geom, const pa_balls *balls, int32_t n_frames,
                               unsigned long long *out, void *stream);

/* One Adam step on a device float array (the paper's optimiser is not named;
 * Sec. 3.2 gives per-group learning rates and a step decay):
 *   m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 *   x -= lr * (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * x, g, m, v device [n], 16-byte aligned. step >= 1.  The scalars are host
 * doubles; 1 - b1, 1 - b2 and the bias corrections are formed in double and
 * rounded once to float. */
PA_API int32_t pa_adam_step(float *x, const float *g, float *m, float *v, int64_t n, double lr, double beta1,
                            double beta2, double eps, int32_t step, void *stream);

/* Adam with the step number read from device memory, so that a whole IR
 * iteration can be replayed from one CUDA graph: t = *step (>= 1), learning
 * rate lr0 * gamma^floor((t-1)/step_size) (the step decay of Sec. 3.2:
 * step_size 160, drop rate 0.1), bias corrections 1 - beta^t.  Otherwise as
 * pa_adam_step.  step: device int32. */
PA_API int32_t pa_adam_step_scheduled(float *x, const float *g, float *m, float *v, int64_t n, double lr0,
                                      double beta1, double beta2, double eps, int32_t step_size, double gamma,
                                      const int32_t *step, void *stream);

/* Adds 1 to the device int32 *step (one-thread kernel, stream ordered). */
PA_API int32_t pa_step_increment(int32_t *step, void *stream);

/* ------------------------------------------------------------------------
 * Imaging (Sec. 3.1-3.2, Tab. 1).  The paper compares 4D SlingBAG with the
 * universal back-projection (UBP), shows maximum amplitude projections (MAPs)
 * of reconstructions converted to voxel grids, and scores them by SSIM; it
 * prints none of these methods, so each call below computes the textbook
 * definition stated with it.
 * ---------------------------------------------------------------------- */

/* UBP filtering step (Xu and Wang): for every trace p(t_k), t_k = t0 + k/fs,
 *   b(t_k) = 2 p(t_k) - 2 t_k dp/dt(t_k),
 * dp/dt by central differences (one-sided at k = 0 and k = T-1).
 * traces, b: device [n_traces][n_samples] (may not alias); n_samples >= 2. */
PA_API int32_t pa_ubp_filter(const float *traces, int64_t n_traces, int32_t n_samples, float fs, float t0,
                             float *b, void *stream);

/* UBP back-projection of filtered traces b (device [n_sensors][n_samples],
 * from pa_ubp_filter) onto `grid`:
 *   vol(r) = sum_s w_s b_s(|r - r_s| / c) / sum_s w_s,
 * w_s = cos(theta_s) / |r - r_s|^2, theta_s the angle between r - r_s and the
 * sensor's inward normal (from r_s towards `center`, host float[3]); sensors
 * with cos(theta_s) <= 0 are left out; b_s is linearly interpolated at the
 * fractional sample (d/c - t0) fs and is 0 outside [0, T-1].  A voxel no
 * sensor faces gets 0.  geom: sensors, c, fs, t0, n_samples (kappa unused).
 * vol: device [nz][ny][nx], overwritten. */
PA_API int32_t pa_ubp(const pa_geom *geom, const float *center, const float *b, const pa_grid *grid, float *vol,
                      void *stream);

/* Ball cloud -> voxel grid (SlingBAG's conversion of its point cloud,
 * Sec. 2.1): vol(r) = sum_b p_b exp(-|r - mu_b|^2 / (2 a_b^2)) over the
 * closed support |r - mu_b| <= kappa a_b (kappa > 0); balls with a <= 0 or
 * p == 0 add nothing.  balls: one frame, device [5][stride]; vol: device
 * [nz][ny][nx], overwritten.  Deterministic: every voxel sums its balls in
 * index order. */
PA_API int32_t pa_splat(const pa_balls *balls, float kappa, const pa_grid *grid, float *vol, void *stream);

/* Maximum amplitude projections of vol (device [nz][ny][nx]): xy [ny][nx]
 * (max over z), yz [nz][ny] (max over x), xz [nz][nx] (max over y); any of
 * the three outputs may be NULL. */
PA_API int32_t pa_map(const float *vol, const pa_grid *grid, float *xy, float *yz, float *xz, void *stream);

/* Workspace bytes pa_ssim needs for H x W images. */
PA_API size_t pa_ssim_workspace_size(int32_t H, int32_t W);

/* Structural similarity (Wang, Bovik, Sheikh, Simoncelli 2004) of images x
 * and y (device [H][W], H, W >= 11): local means, variances and covariance
 * under an 11 x 11 Gaussian window (sigma 1.5, weights summing to 1) at every
 * position where the window fits,
 *   SSIM = (2 mx my + C1)(2 sxy + C2) / ((mx^2 + my^2 + C1)(sx^2 + sy^2 + C2)),
 * C1 = (0.01 L)^2, C2 = (0.03 L)^2 (L > 0, the dynamic range).  With
 * flags = PA_SSIM_MINMAX each image is first mapped to [0, 1] by its own
 * minimum and maximum (reconstructions in arbitrary units against a ground
 * truth) and L = 1.  Writes the mean to *mean (device double) and, if
 * map != NULL, the SSIM map (device [(H-10)][(W-10)]).  workspace: device,
 * pa_ssim_workspace_size bytes, 16-byte aligned. */
PA_API int32_t pa_ssim(const float *x, const float *y, int32_t H, int32_t W, float L, uint32_t flags, float *map,
                       double *mean, void *workspace, size_t workspace_bytes, void *stream);

/* Self-test of failure detection (no counterpart in the paper): launches one
 * block that waits for an mbarrier phase nothing completes, with the same
 * bounded wait that guards every TMA stage of pa_forward, giving up after
 * limit_ns (1e3 <= limit_ns <= 1e9).  The kernel records PA_ERR_TIMEOUT in the
 * device error word (read it with pa_device_error) and exits with nothing in
 * flight, so the context stays usable. */
PA_API int32_t pa_selftest_bounded_wait(uint64_t limit_ns, void *stream);

/* Measurement aid for the roofline denominators (no counterpart in the
 * paper): the throughput of the units that bound the forward and adjoint
 * sample loops, measured on the current device by probe kernels of eight
 * independent dependency chains per thread in one full wave.  out4 (host)
 * receives, per SM and clock, {scalar FP32 FMA lane operations, packed
 * FP32x2 FMA lane operations (two per lane and instruction), SFU base-2
 * exponentials (ex2.approx.ftz.f32)} and the SM clock in MHz that block 0
 * saw during the scalar probe (clock64 over %globaltimer).  Runs about
 * 0.1 s of device time and synchronises `stream`; allocates nothing. */
PA_API int32_t pa_measure_unit_rates(void *stream, double *out4);

#ifdef __cplusplus
}
#endif

#endif /* PA_H */
