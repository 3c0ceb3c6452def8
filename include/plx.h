/*
 * plx.h - C ABI of the B300 (sm_103a) Plenoxel RGB-D renderer.
 *
 * The library renders rays through a sparse voxel grid and differentiates the
 * result, following "RGB-D Mapping and Tracking in a Plenoxel Radiance Field"
 * (arXiv 2307.03404):
 *   - forward render: Sec. 4, Eq. 1 (colour), Eq. 2 (transmittance), Eq. 3
 *     (expected depth), on the grid of Sec. 5.2 (28 values per vertex,
 *     trilinear interpolation);
 *   - mapping adjoint: Sec. 5.2, Eq. 4-11 (loss and its gradient to the grid);
 *   - tracking: Sec. 5.3, Eq. 12-14 and Appendix A (gradient of the rendered
 *     colour and depth with respect to the camera pose), reduced to a
 *     Gauss-Newton system and stepped on SE(3).
 *
 * Conventions common to every call
 *   - Every function returns a plx_status. On failure plx_last_error() gives a
 *     message (thread-local, valid until the next call on the same thread).
 *     No C++ exception crosses this boundary.
 *   - Array pointers are DEVICE pointers owned by the caller unless a comment
 *     says HOST. Descriptor structs (plx_grid_desc, plx_cameras, plx_rays,
 *     plx_render_opts) are HOST memory, read during the call only.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream. Every call is asynchronous on its stream, except
 *     plx_grid_create / plx_grid_destroy / plx_grid_check, which synchronise,
 *     and plx_grid_set_config when it rebuilds the empty-space maps. Besides
 *     those, only plx_grid_grow allocates (stream-ordered scratch), so the
 *     render, backward, pose-step and optimiser calls can be captured in a
 *     CUDA graph.
 *   - A grid handle owns scratch memory: calls that use one handle must not
 *     run concurrently on different streams.
 *
 * Geometry
 *   - Grid: res[0..2] vertices along x, y, z spanning the box [lo, hi];
 *     vertex (x, y, z) sits at lo + (x, y, z) * h with h = (hi - lo)/(res - 1).
 *   - Camera: pinhole, pixel (u, v) has centre (u + 1/2, v + 1/2); camera
 *     frame x right, y down, z forward; pose = camera-to-world [R | o] as a
 *     row-major 3x4 array of doubles. The ray of pixel (u, v) is o + t d with
 *     d = R d_c / |d_c|, d_c = ((u + 1/2 - cx)/fx, (v + 1/2 - cy)/fy, 1).
 *   - Samples: with [t_min, t_max] the overlap of the ray with the grid box
 *     (t_min no smaller than near_t), sample k sits at
 *     t_k = t_min + (k + 1/2) * step for k < floor((t_max - t_min)/step),
 *     at most max_samples; every delta_k is `step`.
 *   - Activations: sigma = max(0, trilinear density); colour = sigmoid (or
 *     identity) of sum_k Y_k(d) * trilinear SH_k, Y the real SH of degree
 *     0..2 in the order (1; y, z, x; xy, yz, 3z^2-1, xz, x^2-y^2).
 *   - Rendered colour includes the background term T_{N+1} * bg.
 *   - Depth targets are sensor z-depths (depth_is_z = 1, converted to ray
 *     distance by |d_c|) or ray distances (depth_is_z = 0). A ray whose depth
 *     target is not positive or not finite is left out of the losses and of
 *     their normaliser M (Sec. 6.1: invalid depth pixels are disregarded).
 */
#ifndef PLX_H
#define PLX_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PLX_OK = 0,
  PLX_EINVAL = 1,        /* bad argument (null pointer, size, range) */
  PLX_ENOMEM = 2,        /* device allocation failed */
  PLX_ECUDA = 3,         /* a CUDA runtime call failed */
  PLX_EDEVICE_CHECK = 4, /* a device-side check failed (see plx_grid_check) */
  PLX_ETIMEOUT = 5,      /* a bounded device wait gave up */
  PLX_EUNSUPPORTED = 6   /* option not supported by this library */
} plx_status;

/* Storage of the 28 values of a vertex inside the library. Every mode
 * computes in FP32; the 16-bit modes halve the bytes gathered per sample. */
typedef enum {
  PLX_STORE_F32 = 0,      /* density and SH in FP32 (128-byte record) */
  PLX_STORE_BF16 = 1,     /* density and SH in BF16 (64-byte record) */
  PLX_STORE_F16 = 2,      /* density and SH in FP16 (64-byte record) */
  PLX_STORE_F32_BF16 = 3  /* density FP32, SH BF16 (64-byte record) */
} plx_storage;

typedef enum { PLX_ACT_SIGMOID = 0, PLX_ACT_IDENTITY = 1 } plx_color_act;

#define PLX_MAX_CAMERAS 128
#define PLX_GRAD_STRIDE 32 /* floats per vertex in gradient buffers */

typedef struct {
  int32_t res[3];     /* vertices along x, y, z; each >= 2 */
  double lo[3];       /* box corner of vertex (0, 0, 0), world units */
  double hi[3];       /* box corner of vertex (res-1), world units; hi > lo */
  int64_t n_alloc;    /* allocated vertices (rows of density / sh) */
  int32_t storage;    /* plx_storage */
  int32_t reserved;
} plx_grid_desc;

typedef struct plx_grid plx_grid; /* opaque */

typedef struct {
  double fx, fy, cx, cy; /* pixels */
  int32_t width, height; /* pixels; width * height < 2^31 */
} plx_intrinsics;

typedef struct {
  int32_t n_cams;              /* 1 .. PLX_MAX_CAMERAS */
  int32_t reserved;
  const plx_intrinsics *intr;  /* HOST [n_cams] */
  const double *poses;         /* DEVICE [n_cams][12] camera-to-world [R | o] */
} plx_cameras;

/* Which rays a call processes.
 * Dense mode (cam_id == NULL and pixel == NULL): every pixel of every camera,
 *   camera after camera, row-major inside a camera; ray index r of pixel
 *   (u, v) of camera c is (sum of W*H of cameras before c) + v*W + u, and
 *   n_rays must be 0 or that total.
 * List mode (pixel != NULL): n_rays rays, ray i is pixel[i] = v*W + u of
 *   camera cam_id[i] (cam_id may be NULL when there is one camera). */
typedef struct {
  int64_t n_rays;
  const int32_t *cam_id; /* DEVICE [n_rays] or NULL */
  const int32_t *pixel;  /* DEVICE [n_rays] or NULL */
} plx_rays;

/* plx_render_opts.pose_flags. PLX_POSE_VIEW_DIR: the pose Jacobian also
 * differentiates the SH colour through the ray direction, dc/dd (a variant:
 * Sec. 5.3 holds the SH direction fixed). Honoured by plx_render_backward_pose,
 * plx_render_backward_pose_noalloc, plx_track_adam_step and the tracking items
 * of plx_render_batch. */
#define PLX_POSE_VIEW_DIR 1

typedef struct {
  double step;         /* sample spacing delta in world units, > 0 */
  double near_t;       /* smallest t marched, >= 0 */
  double stop_T;       /* stop a ray once T_{i+1} < stop_T; 0 = never */
  float bg[3];         /* background colour */
  float lambda_d;      /* lambda_d of Eq. 11, >= 0 */
  int32_t max_samples; /* cap on samples per ray, >= 0 */
  int32_t color_act;   /* plx_color_act */
  int32_t depth_is_z;  /* 1: depth targets are z-depths; 0: ray distances */
  int32_t pose_flags;  /* 0, or PLX_POSE_VIEW_DIR (pose calls only) */
  void *sample_cache;  /* DEVICE, 16-byte aligned, or NULL: the sample cache
                          of plx_render_forward / plx_render_backward_grid
                          (ignored by every other call) */
  int32_t sample_cap;  /* K: samples kept per ray in sample_cache, >= 0 */
  int64_t sample_rays; /* n: rays the cache was sized for (its row stride),
                          >= the call's n_rays */
  int32_t *ray_range;  /* DEVICE int32 [n_rays][2], or NULL: each ray's
                          compositing range (below), written by
                          plx_render_forward and read by the re-marching
                          adjoint of plx_render_backward_grid (ignored by
                          every other call) */
} plx_render_opts;

/* Compositing range (Sec. 5.2: the adjoint recomputes T_i and the prefix sums
 * of Eq. 9-10 front to back). With opts->ray_range set, plx_render_forward
 * writes for ray r (its output row) the sample index of its first sample with
 * sigma > 0 at [r][0] and one past its last at [r][1] (0, 0 when it has none),
 * and plx_render_backward_grid re-marches each ray only over that range. No
 * sample outside it composites, so where the range starts T = 1 and the
 * prefix sums are 0, and the gradients are those of the full re-march (the
 * same products; only the order of the atomic sums differs). It is the
 * per-ray state a recomputing adjoint keeps (8 bytes per ray), and it also
 * shortens the re-march of rays that overflow a sample cache. The adjoint
 * call must name the same array, grid contents, cameras, rays and opts as the
 * forward that wrote it (nothing checks this). With it, calls of at most
 * seg_rays rays also run one ray per lane (plx_launch_config). */

/* Sample cache (Sec. 5.2: what the adjoint of Eq. 8-10 needs per sample).
 * With opts->sample_cache set and opts->sample_cap = K > 0, plx_render_forward
 * keeps, for each ray, its first K samples with sigma > 0 (the ones that
 * composite): the sample index k, the density before the ReLU and the
 * activated colour. plx_render_backward_grid then visits only those samples
 * (no empty-space march, no record gathers, no SH projection; it still loads
 * the cells' links to scatter into the corners) and re-marches in full only
 * the rays that had more than K. Layout, n = opts->sample_rays:
 *   float [K][n][4]  (sigma, c_r, c_g, c_b) of kept sample j of ray r at [j][r]
 *   int32 [K][n]     its sample index k
 *   int32 [n]        the ray's number of samples with sigma > 0 (may exceed K)
 * in plx_sample_cache_bytes(n, K) bytes, owned by the caller, used by one
 * call at a time (calls that share a cache must not run concurrently); a call
 * over more than n rays fails with PLX_EINVAL. The adjoint
 * call must name the same cache and K, grid contents, cameras, rays and opts
 * as the forward that filled it (nothing checks this); without a cache it
 * re-marches every ray. Both ways give the same gradients up to the order of
 * floating-point sums.
 * plx_render_batch uses the same layout with thread slots for rows: a mapping
 * ray keeps its samples in the row of the thread that marches it, between
 * that thread's forward and adjoint, and threads at or past sample_rays
 * re-march. At most 2 x 256 threads per SM are resident in that launch, so
 * sample_rays = 512 x (SM count) covers every thread. */
int64_t plx_sample_cache_bytes(int64_t n_rays, int32_t cap); /* -1 if either < 0 */

const char *plx_last_error(void);
const char *plx_version(void);

/* Sec. 5.2 (model representation), Sec. 6.1 (sparse grid up to 512^3).
 * Copies a grid given in the canonical layout into library-owned device
 * memory in the storage format desc->storage (16-bit modes round to nearest
 * even), builds the empty-cell occupancy it marches with, and checks every
 * link.
 *   links   DEVICE int32 [res_z][res_y][res_x]; -1 or 0 .. n_alloc-1
 *   density DEVICE float [n_alloc]
 *   sh      DEVICE float [n_alloc][27], channel-major (R0..R8, G0..G8, B0..B8)
 * Synchronises `stream`. Errors: PLX_EINVAL (descriptor, or a link out of
 * range), PLX_ENOMEM (also, before anything is allocated, when the
 * environment variable PLX_ALLOC_CAP_BYTES is set below the bytes the grid
 * needs), PLX_ECUDA. On success *out owns the copy; the caller's
 * arrays may be freed. */
plx_status plx_grid_create(const plx_grid_desc *desc, const int32_t *links,
                           const float *density, const float *sh, void *stream,
                           plx_grid **out);

/* Replace every density / SH value (same layout as plx_grid_create; links
 * unchanged), e.g. after an optimiser step. Asynchronous. */
plx_status plx_grid_upload(plx_grid *grid, const float *density,
                           const float *sh, void *stream);

/* Copy the stored values back to the canonical layout (FP32; 16-bit storage
 * is widened exactly). Asynchronous. */
plx_status plx_grid_download(const plx_grid *grid, float *density, float *sh,
                             void *stream);

/* Descriptor of a grid (HOST out). */
plx_status plx_grid_info(const plx_grid *grid, plx_grid_desc *out);

/* Frees the grid's device memory (synchronises the device first). */
plx_status plx_grid_destroy(plx_grid *grid);

/* Sec. 4, Eq. 1-3. Renders every ray of `rays`.
 *   rgb_out   DEVICE float [n_rays][3]  rendered colour C (incl. background)
 *   depth_out DEVICE float [n_rays]     expected depth D (ray distance)
 *   state_out DEVICE float [n_rays]     final transmittance T_{N+1}, or NULL
 *   counts_out DEVICE int32 [n_rays][2] samples marched and samples with an
 *             allocated corner, or NULL (counting costs a little time)
 * With opts->sample_cache it also fills the sample cache (see above).
 * Output row r is ray r (see plx_rays). Errors: PLX_EINVAL (also a sample
 * cache that is not 16-byte aligned), PLX_ECUDA. */
plx_status plx_render_forward(const plx_grid *grid, const plx_cameras *cams,
                              const plx_rays *rays, const plx_render_opts *opts,
                              float *rgb_out, float *depth_out, float *state_out,
                              int32_t *counts_out, void *stream);

/* Sec. 5.2, Eq. 4-11. Mapping adjoint: for the loss
 *   L = 1/M sum_valid |C - C_t|^2 + lambda_d/M sum_valid (D - D_t)^2
 * re-marches every valid ray (or, with a sample cache, visits the samples the
 * forward kept), recomputes T_i and the prefix sums of Eq. 9-10, and ADDS
 * dL/d(value) into `grad`. With grad NULL only (L, M) is computed (no march,
 * no sample cache read): the loss of a forward without its gradient.
 *   rgb_target   DEVICE float [n_rays][3]
 *   depth_target DEVICE float [n_rays] (see depth_is_z)
 *   rgb, depth   DEVICE float, the outputs of plx_render_forward for the
 *                same grid, cameras, rays and opts
 *   grad         DEVICE float [n_alloc][PLX_GRAD_STRIDE], 16-byte aligned:
 *                slot 0 = dL/d density, slots 1..27 = dL/d SH (canonical
 *                order), slots 28..31 untouched. The caller zeroes it. NULL:
 *                loss only.
 *   loss_out     DEVICE double [2] or NULL: overwritten with (L, M).
 * Errors: PLX_EINVAL (also grad and loss_out both NULL), PLX_ECUDA. */
plx_status plx_render_backward_grid(const plx_grid *grid,
                                    const plx_cameras *cams,
                                    const plx_rays *rays,
                                    const plx_render_opts *opts,
                                    const float *rgb_target,
                                    const float *depth_target, const float *rgb,
                                    const float *depth, float *grad,
                                    double *loss_out, void *stream);

/* Sec. 5.3, Eq. 12-14, Appendix A. Tracking: for the rays of camera `cam`
 * (dense mode: all its pixels; list mode: pixel[] of that camera, cam_id
 * ignored) computes the 4x6 Jacobian of (C - C_t, D - D_t) with respect to
 * a left perturbation xi = (rho, phi) of the pose, T <- exp(xi^) T, with t_i,
 * delta_i and the SH direction held fixed as in the paper, and reduces it in
 * FP64 over the valid rays with W = diag(1, 1, 1, lambda_d) / M:
 *   JtWJ DEVICE double [36] = sum J^T W J (row-major, symmetric)
 *   JtWr DEVICE double [6]  = sum J^T W r
 *   loss DEVICE double [2]  = (sum r^T W r, M)
 * All three are overwritten. The reduction order is fixed, so the result is
 * deterministic. Targets are indexed like the rays. */
plx_status plx_render_backward_pose(const plx_grid *grid,
                                    const plx_cameras *cams, int32_t cam,
                                    const plx_rays *rays,
                                    const plx_render_opts *opts,
                                    const float *rgb_target,
                                    const float *depth_target, double *JtWJ,
                                    double *JtWr, double *loss, void *stream);

/* Allocation-free variant of plx_render_backward_pose. The paper has no
 * counterpart. It serves callers that cannot allocate device memory while
 * they run, so cannot call plx_grid_create: a tracking loop under a real-time
 * budget that forbids allocation after start-up, or an application whose
 * device memory all belongs to another allocator (a pool this library cannot
 * see). The caller passes the grid as plain arrays instead of a handle:
 *   desc    HOST descriptor (res, lo, hi, n_alloc, storage)
 *   links   DEVICE int32 [res_z][res_y][res_x]; each entry -1 or in
 *           [0, n_alloc). NOT checked here (plx_grid_create checks them).
 *   records DEVICE, 32-byte aligned, one record per allocated vertex in the
 *           layout of desc->storage: PLX_STORE_F32 = 32 floats (slot 0
 *           density, slots 1..27 SH in canonical order, 28..31 ignored);
 *           PLX_STORE_BF16 / PLX_STORE_F16 = 32 16-bit values in the same
 *           slots; PLX_STORE_F32_BF16 = 64 bytes, density as float in bytes
 *           0..3, the 27 SH as bfloat16 from byte 4.
 * Every other argument and all outputs are those of plx_render_backward_pose.
 * Scratch: a static device array inside the library holding the FP64 partial
 * sums of at most 1024 thread blocks (about 256 KiB), kept by every GPU that
 * loads the library until the process exits. The kernel strides over ray
 * tiles with at most that many blocks, so every ray count fits; a device
 * index of 64 or more is rejected with PLX_EUNSUPPORTED. The first call on a
 * device looks up the array's device address with that device current: make
 * that first call before any stream capture. All calls share the array, and
 * each call clears its counters on its own stream first: calls that overlap
 * on the GPU (several streams or host threads) race and return wrong sums.
 * Pixel-list entries out of range are skipped and do not count in M
 * (plx_noalloc_error reports them). Nothing is allocated or freed. */
plx_status plx_render_backward_pose_noalloc(
    const plx_grid_desc *desc, const int32_t *links, const void *records,
    const plx_cameras *cams, int32_t cam, const plx_rays *rays,
    const plx_render_opts *opts, const float *rgb_target,
    const float *depth_target, double *JtWJ, double *JtWr, double *loss,
    void *stream);

/* The error word of the last plx_render_backward_pose_noalloc call on the
 * current device, copied on `stream` into err_out (DEVICE or HOST int32 [1];
 * nothing is allocated): 0, or bit 0 set when the pixel list held entries
 * out of range (skipped, not counted in M). Enqueue it on the call's stream
 * before the next call clears the word; calls that overlap race as described
 * above. Errors: PLX_EINVAL (null err_out, or no call on this device yet),
 * PLX_EUNSUPPORTED, PLX_ECUDA. */
plx_status plx_noalloc_error(int32_t *err_out, void *stream);

/* Sec. 5.3 (the pose is optimised directly). Gauss-Newton step, on the
 * device in FP64: solves (JtWJ + damping I) xi = -JtWr by Cholesky and sets
 * pose <- exp(xi^) pose (SE(3) exponential: Rodrigues rotation, V rho
 * translation).
 *   pose    DEVICE double [12], updated in place (e.g. plx_cameras.poses + 12c)
 *   xi_out  DEVICE double [6] or NULL
 *   status  DEVICE int32 [1] or NULL: 0, or 1 when the damped system is not
 *           positive definite (the pose is then left unchanged)
 * Asynchronous; graph-capturable. */
plx_status plx_pose_step(const double *JtWJ, const double *JtWr, double damping,
                         double *pose, double *xi_out, int32_t *status,
                         void *stream);

/* Sec. 5.3 with Marquardt's damping (the paper optimises the pose with Adam,
 * Sec. 5.4; a plain Gauss-Newton step can overshoot where the density ramps
 * are steep). One call per Jacobian evaluation at the current pose, passing
 * that pose's system and loss:
 *   - the current pose is accepted if this is the first call (state[2] == 0)
 *     or its loss is not above the last accepted one; lambda /= factor (not
 *     below 1e-12, and lambda = lambda_init on the first call);
 *   - otherwise the last accepted pose is restored, lambda *= factor (not
 *     above 1e12), and its system is used instead;
 *   - then (H + lambda (diag H + 1e-12 max diag H)) xi = -b is solved by
 *     Cholesky in FP64 (lambda grows by factor up to 8 times while that is not
 *     positive definite) and pose <- exp(xi^) pose.
 *   JtWJ, JtWr, loss  DEVICE, as written by plx_render_backward_pose
 *   state   DEVICE double [64], zeroed by the caller before the first call:
 *           [0] lambda, [1] loss of the accepted pose, [2] calls made, [3] 1
 *           if this call accepted, [4..15] accepted pose, [16..51] its H,
 *           [52..57] its b
 *   pose    DEVICE double [12], updated in place
 *   xi_out  DEVICE double [6] or NULL; status DEVICE int32 [1] or NULL: 0
 *           accepted, 2 rejected and restored, 1 no damping made the system
 *           definite (pose left at the accepted one)
 * Asynchronous; graph-capturable. Errors: PLX_EINVAL (lambda_init < 0,
 * factor <= 1, null pointers). */
plx_status plx_pose_step_lm(const double *JtWJ, const double *JtWr,
                            const double *loss, double *state,
                            double lambda_init, double factor, double *pose,
                            double *xi_out, int32_t *status, void *stream);

/* Sec. 5.4 (RMSProp for the mapping). One RMSProp step on every stored grid
 * value, in place, from the gradient left by plx_render_backward_grid:
 *   v <- alpha v + (1 - alpha) g^2,  value <- value - lr g / (sqrt(v) + eps)
 * with lr = lr_density for the density and lr_sh for the 27 SH values (the
 * two differ by orders of magnitude in scale; the paper gives no rates),
 * computed in FP32 and stored in the grid's storage format (16-bit formats
 * round to nearest even).
 *   grad   DEVICE float [n_alloc][PLX_GRAD_STRIDE], slots 0..27; set to zero
 *          by the call when zero_grad != 0 (ready for the next adjoint)
 *   state  DEVICE float [n_alloc][PLX_GRAD_STRIDE]: the running v, zeroed by
 *          the caller before the first step
 * Asynchronous; graph-capturable. Errors: PLX_EINVAL. */
plx_status plx_grid_rmsprop(plx_grid *grid, float *grad, float *state,
                            float lr_density, float lr_sh, float alpha,
                            float eps, int32_t zero_grad, void *stream);

/* Sec. 5.3-5.4 (tracking by random rays of the current image, Adam). One
 * iteration on camera `cam`: n_rays pixels drawn from the frame with the
 * counter-based generator SplitMix64 (Steele, Lea and Flood 2014; ray i of
 * iteration t is pixel mix(seed + (t n_rays + i + 1) * 0x9E3779B97F4A7C15)
 * mod (W H), pixels may repeat), their pose system as in
 * plx_render_backward_pose (written to JtWJ, JtWr, loss), the loss gradient
 * g = 2 JtWr with respect to a left perturbation, and an Adam step
 *   m <- b1 m + (1 - b1) g,  v <- b2 v + (1 - b2) g^2,
 *   xi = -lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),
 *   pose <- exp(xi^) pose   (cams->poses row `cam`, in place).
 *   rgb_target, depth_target  DEVICE, the whole frame: [W*H][3], [W*H]
 *   state  DEVICE double [20]: m[0..5], v[6..11], t at [12] (iterations done,
 *          also the generator counter), last xi at [13..18]; zeroed by the
 *          caller before the first iteration.
 * Up to 8192 rays per iteration are drawn by a separate one-block kernel and
 * launched in the Z-order of their pixels (the same set; only the order in
 * which warps take them, and so the summation order, changes).
 * Asynchronous; graph-capturable (the counter lives on the device). */
plx_status plx_track_adam_step(const plx_grid *grid, const plx_cameras *cams,
                               int32_t cam, const plx_render_opts *opts,
                               int32_t n_rays, uint64_t seed,
                               const float *rgb_target,
                               const float *depth_target, double *state,
                               double lr, double beta1, double beta2,
                               double eps, double *JtWJ, double *JtWr,
                               double *loss, void *stream);

/* Sec. 6.1 (the paper maps into "a dynamic voxel grid" and does not say how
 * it grows). Growth from observed depth, on the caller's link array: every
 * pixel whose depth is positive and finite is lifted to its surface point
 *   X = o + s R d_c,  d_c = ((u + 1/2 - cx) / fx, (v + 1/2 - cy) / fy, 1),
 *   s = z (depth_is_z != 0, z-depth) or z / |d_c| (ray distance),
 * and every vertex i with |i_a - (X_a - lo_a) / h_a| <= band on each axis a
 * is allocated if it was not. The new vertices get the numbers n_alloc,
 * n_alloc + 1, ... in link order (x fastest, then y, then z), whatever the
 * order in which pixels run. The per-pixel arithmetic is FP64, each
 * operation rounded once, in the order written above.
 *   desc   HOST: res, lo, hi and n_alloc (the current count); storage unused
 *   links  DEVICE int32 [res_z][res_y][res_x], -1 or 0 .. n_alloc-1 (the value
 *          -2 is reserved); updated in place
 *   cams   intrinsics HOST, poses DEVICE (camera-to-world)
 *   depth  DEVICE float [sum of W*H]: every pixel of every camera, camera
 *          after camera, row-major
 *   band   0 .. 16 (grid units)
 *   n_new  DEVICE int64 [1]: vertices added, or -1 if n_alloc + added would
 *          exceed INT32_MAX (then links is left as it was)
 * Asynchronous (uses stream-ordered scratch of 8 bytes per 4096 vertices).
 * A grid handle built on the old links does not see the change: create a new
 * one with the grown links and values. Errors: PLX_EINVAL, PLX_ENOMEM,
 * PLX_ECUDA (links may then hold -2 marks). */
plx_status plx_grid_grow(const plx_grid_desc *desc, int32_t *links,
                         const plx_cameras *cams, const float *depth,
                         int32_t depth_is_z, double band, int64_t *n_new,
                         void *stream);

/* Launch choices of a grid's kernels (the paper has none; they do not change
 * any result). block_shift: the empty-space map marks blocks of
 * 2^block_shift cells per axis (1..6); rays jump over blocks without an
 * allocated vertex. fine_skip: a second level inside non-empty blocks (blocks
 * of 2 cells per axis), per kernel: bit 0 forward, 1 grid adjoint, 2 pose
 * Jacobian, 3 batched launch (PLX_FINE_*). *_blocks: each ray kernel is compiled for 1 or 2
 * resident blocks of 256 threads per SM (a register budget of 255 or 128 per
 * thread): forward, grid adjoint, pose Jacobian, batched launch; the forward
 * also for 3 (80 registers). seg_rays: rays per warp. A call over at most
 * seg_rays rays (ray slots: dense frames count whole 8x4 tiles) runs a warp
 * per ray in the forward, the re-marching grid adjoint and the pose Jacobian
 * (the 32 lanes split each ray's samples and a scan combines the segments;
 * only without early stop, sample cache or view-direction term, and for the
 * sigmoid colour), larger calls one ray per lane; 0 = always one ray per
 * lane; at most 2^24. Defaults are
 * the best measured on B300 for room-scale grids; the Python autotuner times
 * the alternatives on a caller's workload. */
#define PLX_FINE_FORWARD 1
#define PLX_FINE_ADJOINT 2
#define PLX_FINE_POSE 4
#define PLX_FINE_BATCH 8

typedef struct {
  int32_t block_shift;
  int32_t forward_blocks;
  int32_t adjoint_blocks;
  int32_t pose_blocks;
  int32_t batch_blocks;
  int32_t fine_skip;
  int32_t seg_rays;
} plx_launch_config;

/* Current launch choices of a grid (HOST out). */
plx_status plx_grid_get_config(const plx_grid *grid, plx_launch_config *out);

/* Sets the launch choices. A new block_shift or fine_skip rebuilds the
 * empty-space maps (allocates, synchronises `stream`); otherwise nothing runs
 * on the device.
 * Errors: PLX_EINVAL (out of range), PLX_ENOMEM, PLX_ECUDA. */
plx_status plx_grid_set_config(plx_grid *grid, const plx_launch_config *config,
                               void *stream);

/* Kinds of work in a batch. */
typedef enum { PLX_WORK_MAP = 0, PLX_WORK_TRACK = 1 } plx_work_mode;

typedef struct {
  int32_t cam;  /* camera index in plx_cameras (a camera may appear more than once) */
  int32_t mode; /* plx_work_mode */
} plx_work;

/* Sec. 5.2 + Sec. 5.3 in one persistent launch: frames of any sizes, some to
 * map (forward, loss and adjoint to the grid, as plx_render_forward followed
 * by plx_render_backward_grid) and some to track (as
 * plx_render_backward_pose), processed by one kernel that pulls 32-ray tiles
 * from a global counter, mapping tiles first.
 *   work         HOST [n_work], 1 <= n_work <= PLX_MAX_CAMERAS
 *   rgb_target   DEVICE float [rows][3], depth_target DEVICE float [rows]:
 *                every pixel of every item, item after item in the order of
 *                `work`, row-major inside an item
 *   grad         DEVICE float [n_alloc][PLX_GRAD_STRIDE], 16-byte aligned:
 *                ADDS dL/d(value) of the mapping loss over all mapping items
 *                (one M over all of them); may be NULL without mapping items
 *   map_loss     DEVICE double [2] or NULL: overwritten with (L, M)
 *   JtWJ, JtWr, track_loss  DEVICE double [n_track][36], [n_track][6],
 *                [n_track][2], n_track = number of tracking items, in their
 *                order in `work`; overwritten; may be NULL without tracking
 *                items. Each item's sums are FP64; the order in which tiles
 *                add into them varies between runs (last-bit differences).
 * Errors: PLX_EINVAL, PLX_ECUDA. */
plx_status plx_render_batch(const plx_grid *grid, const plx_cameras *cams,
                            const plx_work *work, int32_t n_work,
                            const plx_render_opts *opts, const float *rgb_target,
                            const float *depth_target, float *grad,
                            double *map_loss, double *JtWJ, double *JtWr,
                            double *track_loss, void *stream);

/* Measurement kernels for the rooflines of the mapping kernels (the paper has
 * none). The grid adjoint scatters each corner's 28 gradient values as 7
 * float4 reductions into the vertex's 128-byte gradient row and the forward
 * gathers 64- or 128-byte vertex records; both run mostly in L2, so their
 * bound is the rate L2 sustains for such accesses, which these kernels issue
 * with nothing else around them (time a launch with CUDA events):
 *   PLX_PROBE_RED     each thread, `ops` times: a row drawn at random from
 *                     n_rows (lanes in groups of `group` share it), 7 float4
 *                     atomic adds of 1e-7 into its floats 0..27;
 *                     7 * ops * threads reductions per launch
 *   PLX_PROBE_GATHER  the same rows, 7 float4 loads each (read only)
 *   PLX_PROBE_STREAM  `ops` coalesced float4 passes over all rows (read only)
 *   PLX_PROBE_RED_ROWS the same rows and additions as PLX_PROBE_RED, sent
 *                     the way the sample-cache adjoint sends them: a warp
 *                     instruction covers 4 rows, 7 lanes per row with one
 *                     float4 each (one coalesced request per row);
 *                     ops * threads rows per launch ('group' is ignored)
 *   PLX_PROBE_ISSUE   instruction issue instead of memory: each thread, `ops`
 *                     times, 512 FP32 fused multiply-adds in 8 independent
 *                     chains (64 per chain), so the SM sub-partitions issue
 *                     back to back; 512 * ops * threads / 32 warp FMA
 *                     instructions per launch (plus a few per `ops` round
 *                     for the loop). buf is written only if a chain ends at
 *                     a value the finite inputs cannot reach ('group' and
 *                     n_rows >= 1 as above, otherwise unused)
 *   buf     DEVICE float [n_rows][PLX_GRAD_STRIDE], 16-byte aligned, holding
 *           finite values (RED adds to them); 1 <= n_rows < 2^32
 *   blocks  thread blocks of 256 threads (1 .. 2^20); ops 1 .. 1024;
 *           group 1 .. 32 (ignored by STREAM and RED_ROWS)
 * Asynchronous. Errors: PLX_EINVAL, PLX_ECUDA. */
#define PLX_PROBE_RED 0
#define PLX_PROBE_GATHER 1
#define PLX_PROBE_STREAM 2
#define PLX_PROBE_RED_ROWS 3
#define PLX_PROBE_ISSUE 4
plx_status plx_probe(int32_t kind, float *buf, int64_t n_rows, int32_t group,
                     int32_t ops, int32_t blocks, void *stream);

/* Reads and clears the grid's device error word (synchronises `stream`).
 * Returns PLX_EDEVICE_CHECK if a device-side check failed since the last
 * call. */
plx_status plx_grid_check(const plx_grid *grid, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PLX_H */
