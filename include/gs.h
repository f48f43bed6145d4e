/*
 * gs.h -- C ABI of the GB300 differentiable tile rasterizer (libgs.so).
 *
 * The paper trains 3D Gaussian Splatting primitives, initialised from an
 * isosurface point cloud, to match images rendered from a structured camera
 * orbit (Section III, "Method Overview"); every training view runs the
 * differentiable tile rasterizer of 3D-GS (Section I): EWA projection of the
 * Gaussians, duplication into 16x16 screen tiles, a radix sort on
 * (tile, depth) keys, front-to-back alpha compositing per tile, its
 * reverse-order backward pass and an Adam update.  This header exposes those
 * steps one call each.
 *
 * Conventions shared by every call
 *  - All pointers named "device" are CUDA device pointers on the context's
 *    device; "host" pointers are ordinary host memory.  No call takes
 *    ownership of a caller pointer.
 *  - Calls are asynchronous on the context's stream (gs_set_stream) unless
 *    stated otherwise.  Errors detected on the host (bad arguments, missing
 *    preceding step, allocation failure, CUDA launch errors) are returned
 *    immediately and nothing is launched.  Errors detected on the device
 *    (instance capacity exceeded, a bounded wait that ran out) are recorded
 *    in a device status word and returned by gs_sync.
 *  - Parameters (gs_params) are FP32 "SoA planes": data[p * stride + i] is
 *    plane p of Gaussian i, with
 *        planes 0-2   mean x, y, z (world)
 *        planes 3-5   log-scale s0, s1, s2
 *        planes 6-9   rotation quaternion w, x, y, z (need not be unit)
 *        plane  10    opacity logit o (opacity = 1 / (1 + exp(-o)))
 *        planes 11..  SH colour coefficients, plane 11 + 3k + c = coefficient
 *                     k (k = l*l + l + m, real orthonormal basis) of channel c
 *    P = 11 + 3 (deg+1)^2 planes; stride >= n, stride % 4 == 0, data 16-byte
 *    aligned.  Gradients and Adam moments use the same layout.
 *  - Images are FP32, planar, [view][channel 3][height][width], the views of
 *    a batch concatenated in order (view v starts at 3 * sum_{u<v} W_u H_u).
 *  - One context serves one host thread at a time.
 */
#ifndef GS_H
#define GS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  GS_OK = 0,
  GS_EINVAL = 1,     /* bad argument; nothing launched */
  GS_ENOMEM = 2,     /* device allocation failed */
  GS_ECUDA = 3,      /* CUDA runtime error (message in gs_last_error) */
  GS_ECAPACITY = 4,  /* more tile instances than the preset capacity */
  GS_ETIMEOUT = 5,   /* a bounded device-side wait ran out */
  GS_EBUSY = 6,      /* server: no free slot / memory budget */
  GS_EAGAIN = 7,     /* server: result not ready before the timeout */
  GS_ESTATE = 8      /* a call needs a preceding step that has not run */
} gs_status;

typedef struct gs_ctx gs_ctx;

/* Context limits.  Zero fields take defaults (see gs_create). */
typedef struct {
  int64_t max_gaussians;     /* N capacity for workspaces (grown on demand) */
  int32_t max_views;         /* views per batch, <= 64 */
  int32_t flags;             /* reserved, 0 */
  int64_t instance_capacity; /* 0: grow on demand (host reads the count);
                                > 0: fixed capacity, overflow -> GS_ECAPACITY
                                (required for CUDA-graph capture) */
} gs_config;

/* Pinhole camera, world -> camera.  The camera looks down +z, x right,
 * y down; pixel (i, j) is the point (i, j) of the image plane, so the
 * principal point of a centred camera is ((W-1)/2, (H-1)/2). */
typedef struct {
  float viewmat[16]; /* row-major 4x4 world->camera (rotation rows, translation column) */
  float fx, fy, cx, cy;
  int32_t width, height;
  float znear;       /* Gaussians with depth <= znear are culled */
  float bg[3];       /* background colour composited behind the Gaussians */
} gs_camera;

/* A Gaussian set (device) in the plane layout above. */
typedef struct {
  float* data;
  int64_t n;
  int64_t stride;
  int32_t sh_degree; /* 0..3 */
  int32_t reserved;
} gs_params;

/* Adam hyper-parameters: one learning rate per parameter group.  flags:
 * GS_ADAM_SQRT_BATCH_LR multiplies every learning rate by sqrt(B), B = views
 * of the context's last projected batch (the learning-rate scaling batched
 * 3D-GS trainers such as Grendel-GS apply; off by default).
 * GS_ADAM_VISIBLE_ONLY is the sparse (visible-only) variant 3D-GS trainers
 * use: a Gaussian that touches no tile in any view of the context's last
 * projected batch keeps its parameters and both moments unchanged (no decay);
 * every other Gaussian takes the usual step, bias-corrected by the global
 * step count.  Off by default: it changes the optimisation trajectory. */
typedef struct {
  float lr_mean, lr_scale, lr_quat, lr_opacity, lr_sh_dc, lr_sh_rest;
  float beta1, beta2, eps;
  int32_t flags;
} gs_adam_hp;

enum { GS_ADAM_SQRT_BATCH_LR = 1, GS_ADAM_VISIBLE_ONLY = 2 };

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device`.  cfg may be NULL (defaults:
 * max_views 64, instance capacity grown on demand).  Allocates the device
 * status word; workspaces are allocated lazily and grow.  *out is NULL on
 * error.  Errors: GS_EINVAL (out NULL, bad cfg), GS_ECUDA, GS_ENOMEM. */
gs_status gs_create(gs_ctx** out, int device, const gs_config* cfg);

/* Free every device buffer of the context (synchronises its stream). */
void gs_destroy(gs_ctx* ctx);

/* Last error message of this context ("" when none); owned by the context. */
const char* gs_last_error(const gs_ctx* ctx);

/* Use `stream` (a cudaStream_t, NULL = legacy default stream) for every
 * following call of this context. */
gs_status gs_set_stream(gs_ctx* ctx, void* stream);

/* Wait for the context's stream; return the device status word (GS_OK,
 * GS_ECAPACITY or GS_ETIMEOUT) and clear it.  After GS_ETIMEOUT or
 * GS_ECAPACITY the sorted keys, values and ranges of the batches since the
 * previous gs_sync, and everything computed from them (images, T_final,
 * gradients, an Adam step taken on those gradients), are undefined; every
 * kernel stays within its buffers on such data, and the next sort that
 * completes is correct again.  A sort partition that gives up its bounded
 * look-back marks itself failed, and every later partition of the same pass
 * gives up on seeing that mark instead of scattering with a partial offset. */
gs_status gs_sync(gs_ctx* ctx);

/* Tunable options of a context (the autotuner sets these). */
typedef enum {
  GS_OPT_RASTER_FWD = 0, /* forward compositing kernel: 1, 2 or 4 = pixels per
                            thread with one block per tile, 8 = one warp per
                            tile.  All variants give the same result up to
                            FP32 rounding. */
  GS_OPT_RASTER_BWD = 1, /* backward compositing kernel, same values */
  GS_OPT_BWD_DIRECT = 2, /* backward: a warp whose pixels meet a Gaussian in at
                            most this many lanes (0..32, default 2) adds the
                            lanes' gradients with per-lane atomics instead of
                            a warp reduction.  Same result up to FP32
                            summation order. */
  GS_OPT_SORT_ITEMS = 3, /* keys per thread of a radix-sort partition: 12, 16
                            (default), 20 or 24 (partitions of 256 x items
                            keys).  Same result.  Fixed once a training graph
                            is captured (GS_ESTATE). */
  GS_OPT_SORT_WAIT = 4,  /* look-back rounds a radix-sort partition waits for
                            the partitions before it: 1 .. 1048576 (default
                            1048576, about a second), after which the sort
                            gives up and the next gs_sync reports
                            GS_ETIMEOUT.  0: every partition that has to look
                            back gives up at once (exercises the timeout
                            path; the blocks return, nothing hangs).  Fixed
                            once a training graph is captured (GS_ESTATE). */
  GS_OPT_TILE_ORDER = 5  /* order in which the compositing kernels take the
                            batch's tiles: 0 (default) bin order; 1 longest
                            lists first (tiles bucketed by floor(log2(list
                            length + 1)), bin order within a bucket; one extra
                            sort pass over the bins per batch).  Same result
                            (the fused L1 loss sums its per-tile partials in
                            bin order either way).  Fixed once a training graph
                            is captured (GS_ESTATE). */
} gs_option;

/* Set / read an option.  Errors: GS_EINVAL (unknown option, bad value). */
gs_status gs_set_option(gs_ctx* ctx, int32_t option, int64_t value);
gs_status gs_get_option(gs_ctx* ctx, int32_t option, int64_t* value);

/* ---------------------------------------------------------------- the path */

/* Step 1, projection (EWA splatting of 3D-GS, Section I; Gaussians from the
 * point cloud, Section III).  For each of the B cameras (host array) and
 * each Gaussian: t = W mu + tau, cull if depth <= znear, Sigma = R S S^T R^T,
 * Sigma' = J W Sigma W^T J^T + 0.3 I (J with image-plane slopes clamped to
 * 1.3x the half field of view), conic = Sigma'^-1, radius
 * ceil(3 sqrt(lambda_max)), the tile rect of that radius, opacity sigma(o)
 * and view-dependent colour max(0, SH(d) + 0.5).  The tiles that receive the
 * Gaussian are those of the rect that the box around its alpha >= 1/255
 * ellipse (half-extents hx, hy of GS_BUF_REC2, the box the compositing
 * passes cull with) reaches: a tile the box misses holds no pixel where the
 * Gaussian could contribute, so leaving it out changes no pixel.  Results
 * stay in the context for the next steps.  1 <= B <= max_views; cameras may
 * differ in resolution.
 * Errors: GS_EINVAL (null pointers, n <= 0, sh_degree outside 0..3, bad
 * stride/alignment, width/height <= 0), GS_ENOMEM, GS_ECUDA. */
gs_status gs_project(gs_ctx* ctx, const gs_params* params, const gs_camera* cams, int32_t B);

/* Step 2, binning (Section I: per-tile lists ordered by depth): each
 * tile's list holds the Gaussians whose tile rect covers it, ordered by
 * (FP32 depth, Gaussian index) -- the order of a stable sort of the 64-bit
 * keys (bin << 32) | depth bits (bin = the view's first tile + ty * gw + tx)
 * of one instance per touched tile.  Computed as: exclusive scans of the
 * per-(view, Gaussian) tile counts and visible flags, a stable LSD onesweep
 * radix sort of each view's visible Gaussians by depth bits, emission of
 * one (bin, Gaussian) instance per touched tile in that order, a stable
 * onesweep sort of the instances by bin, and per-bin [start, end) ranges of
 * the sorted list.  With a grow-on-demand context this call reads the
 * instance count on the host (one stream synchronisation).  Errors:
 * GS_ESTATE (no gs_project), GS_ENOMEM, GS_ECUDA; device-side GS_ECAPACITY
 * and GS_ETIMEOUT via gs_sync. */
gs_status gs_bin_sort(gs_ctx* ctx);

/* Step 3, forward compositing.  Per pixel, over its tile's sorted list:
 * alpha = min(0.99, opacity * exp(power)), skip if power > 0 or
 * alpha < 1/255, stop before a Gaussian that would bring T below 1e-4,
 * C += rgb alpha T, T *= 1 - alpha; output C + T bg.  images: device,
 * [B][3][H][W] as above.  Also keeps, for the backward pass, T_final and the
 * index of the last contributor per pixel, and per tile instance (4 bytes)
 * the 2x4-pixel cells of its tile where it contributed to some pixel.
 * Errors: GS_ESTATE (no gs_bin_sort), GS_EINVAL (images NULL), GS_ECUDA. */
gs_status gs_raster_fwd(gs_ctx* ctx, float* images);

/* gs_raster_fwd and gs_l1_loss(images, targets) in one pass: the compositing
 * kernel also writes dL/dimages = sign(image - target) / count and one
 * partial sum of |image - target| per warp, which a second kernel adds in a
 * fixed order into *loss = mean |image - target| (count = 3 x pixels of the
 * batch).  images may be NULL (not written); targets, loss and dL_dimages:
 * device, image layout.  Same results as the two calls (the loss up to FP32
 * summation order).
 * Errors: GS_ESTATE (no gs_bin_sort), GS_EINVAL (NULL targets, loss or
 * dL_dimages), GS_ECUDA. */
gs_status gs_raster_fwd_l1(gs_ctx* ctx, float* images, const float* targets, float* loss, float* dL_dimages);

/* Step 4, backward.  Given dL/dimages (device, image layout), walks each
 * pixel's tile list in reverse from its last contributor -- only the entries
 * the forward pass recorded as contributing to the pixel's 2x4-pixel cell --
 * recovering T by division, and writes dL/dparams into grads->data (device, overwritten;
 * same n, stride and degree as params).  The derivative is the exact one of
 * step 3 where it exists: zero through a clamped alpha (opacity * G > 0.99),
 * the slope clamp and the colour clamp.  params must be the set given to
 * gs_project.  Errors: GS_ESTATE (no gs_raster_fwd), GS_EINVAL, GS_ECUDA. */
gs_status gs_raster_bwd(gs_ctx* ctx, const gs_params* params, const float* dL_dimages,
                        gs_params* grads);

/* L1 photometric loss over `count` floats (device): *loss = mean |x - y|
 * (device scalar) and dL_dx = sign(x - y) / count (device; sign(0) = 0).
 * Either output may be NULL.  Errors: GS_EINVAL, GS_ECUDA. */
gs_status gs_l1_loss(gs_ctx* ctx, const float* x, const float* y, int64_t count, float* loss,
                     float* dL_dx);

/* L1 loss that allocates no device memory (the paper has no counterpart; this
 * is a service for callers that may not allocate).  Same result as
 * gs_l1_loss: *loss = mean |x - y| and dL_dx = sign(x - y) / count, either
 * output may be NULL.  It exists for callers that cannot call cudaMalloc --
 * an application that gives this library a fixed piece of device memory and
 * forbids further allocation, a render or training loop that must never
 * allocate (an allocation can synchronise the device) once running, a plugin
 * whose host owns all device memory -- so it takes no context (creating one
 * allocates) and keeps its per-block partial sums in a 16 KiB array compiled
 * into the library, present on every GPU that loads the library until the
 * process exits.
 *  - Runs on the calling thread's current CUDA device, on `stream` (a
 *    cudaStream_t, NULL = legacy default stream); x, y, loss and dL_dx are
 *    device pointers on that device.
 *  - The first call on a device looks up the array's device address (set-up,
 *    once per device); make that first call before any stream capture.
 *  - count must be in 1 .. 268,435,456 (4096 partial sums of 65,536
 *    elements); larger counts return GS_EINVAL and launch nothing.
 *  - All calls on a device share the array: calls whose kernels overlap on
 *    the GPU (different streams, no ordering between them) race and give
 *    wrong losses.  Every slot read in a call is written earlier in that same
 *    call, so nothing needs clearing between calls.
 * Errors: GS_EINVAL (x or y NULL, count out of range), GS_ECUDA (set-up or
 * launch failed). */
gs_status gs_l1_loss_noalloc(const float* x, const float* y, int64_t count, float* loss, float* dL_dx,
                             void* stream);

/* D-SSIM training loss of 3D-GS (the paper reports its renders by PSNR and
 * SSIM, Results Tables II-III; the 3D-GS training it runs adds this term):
 * over the views of the context's last projected batch (sizes as given to
 * gs_project), with x = images and y = targets (device, image layout),
 *   *loss = (1 - lambda) mean |x - y| + lambda (1 - mean SSIM)
 * where SSIM is computed per channel with the 11 x 11 Gaussian window
 * (sigma 1.5, zero padding at the image border, weights not renormalised),
 * C1 = 0.01^2, C2 = 0.03^2, and both means run over every (view, channel,
 * pixel).  dL_dimages (device, image layout, overwritten) receives the exact
 * gradient of *loss (sign(0) = 0 in the L1 part).  Either output may be NULL
 * (not both).  lambda = 0.2 is 3D-GS's choice.  Uses 12 bytes of scratch per
 * image element.  Errors: GS_ESTATE (no gs_project), GS_EINVAL, GS_ENOMEM,
 * GS_ECUDA. */
gs_status gs_ssim_loss(gs_ctx* ctx, const float* images, const float* targets, float lambda, float* loss,
                       float* dL_dimages);

/* Quality metrics per view of the last projected batch: ssim[v] = mean SSIM
 * (as in gs_ssim_loss) and psnr[v] = 10 log10(1 / mean (x - y)^2) over view
 * v's channels and pixels (host arrays of B doubles; either may be NULL, not
 * both).  Synchronises the stream.  Errors: as gs_ssim_loss. */
gs_status gs_image_metrics(gs_ctx* ctx, const float* images, const float* targets, double* ssim, double* psnr);

/* Point-cloud initialisation (the paper starts 3D-GS from the isosurface of
 * a volume extracted as a point cloud instead of SfM points, Method
 * Overview).  Isosurface edge crossings of volume (device, float
 * [nz][ny][nx], sample (x, y, z) at origin + spacing * (x, y, z)): for every
 * grid edge whose end values a, b lie on different sides of the level
 * (a >= iso differs from b >= iso), the point at t = (iso - a) / (b - a)
 * along the edge and the volume gradient (central differences, one-sided at
 * the border) interpolated the same way and normalised (pointing towards
 * larger values), in vertex order (x fastest, then y, then z; per vertex its
 * +x, +y, +z edges).  Always sets *count (host) to the number of crossings;
 * with points == normals == NULL it only counts; otherwise points and
 * normals (device, float [capacity][3]) receive them.  Synchronises the
 * stream.  Ends the context's current batch (gs_project must run again).
 * Errors: GS_EINVAL, GS_ECAPACITY (more crossings than capacity; nothing
 * written), GS_ENOMEM, GS_ECUDA. */
gs_status gs_iso_crossings(gs_ctx* ctx, const float* volume, int32_t nx, int32_t ny, int32_t nz, float iso,
                           const float* origin /* host [3] */, const float* spacing /* host [3] */, float* points,
                           float* normals, int64_t capacity, int64_t* count);

/* Initial Gaussians from a point cloud (device, float [m][3] points and unit
 * normals): the n points select[0..n) (device int64 indices into the m, or
 * select == NULL with n == m) become out's n Gaussians: mean = point,
 * log-scales (s, s, s + log flatten) with s = log sqrt of the mean squared
 * distance to the 3 nearest other selected points (exact; floored at 1e-14),
 * the rotation taking +z onto the normal (quaternion (1 + n_z, -n_y, n_x, 0)
 * normalised; (0, 1, 0, 0) for n = -z), opacity logit as given, SH DC
 * 2 sqrt(pi) (c - 1/2) with the Lambertian grey c = 0.1 + 0.9 max(0,
 * n . (1,1,1)/sqrt 3), higher SH 0.  The neighbours are found on the GPU with
 * a uniform grid (points sorted by cell with the binning's radix sort).
 * Synchronises the stream; ends the context's current batch.  Errors:
 * GS_EINVAL (n < 4, n != out->n, m < n, flatten <= 0, points spanning no
 * box), GS_ENOMEM, GS_ECUDA. */
gs_status gs_init_gaussians(gs_ctx* ctx, const float* points, const float* normals, int64_t m, const int64_t* select,
                            int64_t n, float flatten, float opacity_logit, gs_params* out);

/* Adaptive density control of 3D-GS (the paper is silent on it; N is set
 * by the point cloud unless the caller densifies).  gs_set_densify_stats:
 * every following gs_raster_bwd adds, per Gaussian i, to grad_accum[i] the
 * norms of its screen-space mean gradient in normalised device coordinates,
 * ||(dL/dmu2D_x W/2, dL/dmu2D_y H/2)||, over the views of the batch where it
 * touches a tile, and to count[i] the number of those views (device arrays of
 * at least n floats owned by the caller, who zeroes them; both NULL
 * disables; fixed once a training graph is captured).
 * gs_densify writes the new set of one densification step into p_out,
 * m_out, v_out (device, the layout of p, capacity = their common stride; their
 * n is ignored) and *n_out (host) = its size.  For Gaussian i, avg =
 * grad_accum[i] / count[i] (0 when count is 0), smax = largest exp(log-scale):
 *   opacity sigma(o_i) < min_opacity   -> removed;
 *   avg >= grad_threshold and smax <= percent_dense * scene_extent -> kept,
 *     then a copy with zero moments (clone);
 *   avg >= grad_threshold, larger -> replaced by split_n Gaussians with means
 *     mu + R(q/|q|) (exp(s) * z_k), z_k = noise[i][k][0..3) (device, standard
 *     normals the caller draws, [n][split_n][3]), log-scales s - log(0.8
 *     split_n), the other parameters copied, zero moments (split);
 *   otherwise kept with its moments.
 * The outputs keep the input order, a Gaussian's outputs together.
 * Synchronises the stream (reads the new size); ends the context's current
 * batch.  Errors: GS_EINVAL, GS_ECAPACITY (the new set exceeds the output
 * stride; *n_out is set, nothing written), GS_ENOMEM, GS_ECUDA. */
typedef struct {
  float grad_threshold; /* 3D-GS: 0.0002 */
  float percent_dense;  /* 0.01 */
  float scene_extent;   /* world units */
  float min_opacity;    /* 0.005 */
  int32_t split_n;      /* 2 (1..4) */
  int32_t reserved;
} gs_densify_hp;

gs_status gs_set_densify_stats(gs_ctx* ctx, float* grad_accum, float* count);
gs_status gs_densify(gs_ctx* ctx, const gs_params* p, const gs_params* m, const gs_params* v, const float* grad_accum,
                     const float* count, const float* noise, const gs_densify_hp* hp, gs_params* p_out,
                     gs_params* m_out, gs_params* v_out, int64_t* n_out);

/* Step 5, Adam with bias correction (torch.optim.Adam semantics), dense over
 * all planes (or visible-only, see gs_adam_hp), per-group learning rate;
 * step counts from 1.  p, m, v are updated in place; g is read.  All four
 * share n, stride and degree.  Errors: GS_EINVAL (mismatched sets,
 * step < 1), GS_ESTATE (visible-only without a gs_project of a set of the
 * same n and stride), GS_ECUDA. */
gs_status gs_adam(gs_ctx* ctx, gs_params* p, const gs_params* g, gs_params* m, gs_params* v,
                  const gs_adam_hp* hp, int64_t step);

/* ---------------------------------------------------------------- CUDA graph */

/* Capture one whole training step (gs_project, gs_bin_sort, gs_raster_fwd_l1
 * against `targets`, gs_raster_bwd, gs_adam) into a CUDA graph
 * owned by the context, for replay with gs_train_graph_launch.  Needs a
 * context created with a fixed instance_capacity (nothing in the step then
 * reads the device on the host).  Runs the step once uncaptured first (no
 * parameter update) to size every workspace; the capture itself uses a
 * private stream.  Every pointer (parameters, gradients, moments, targets,
 * images, dL/dimages, loss: device) is baked into the graph and must stay
 * valid, except the targets, which each launch names.
 * Errors: GS_EINVAL, GS_ENOMEM, GS_ECUDA, and those of the steps. */
gs_status gs_train_graph_capture(gs_ctx* ctx, gs_params* params, gs_params* grads, gs_params* m, gs_params* v,
                                 const gs_adam_hp* hp, const gs_camera* cams, int32_t B, const float* targets,
                                 float* images, float* dL_dimages, float* loss);

/* Replay the captured step on the context's stream for new cameras (same B
 * and resolutions as captured), the batch's targets (device, image layout)
 * and Adam step number `step` (>= 1).  Cameras, Adam constants and the
 * targets pointer go through a pinned staging area that the graph copies at
 * its start; the call waits (host) until the previous replay has made that
 * copy.  Capacity overflow is reported by gs_sync.
 * Errors: GS_ESTATE (nothing captured), GS_EINVAL (cameras differ, NULL
 * targets), GS_ECUDA. */
gs_status gs_train_graph_launch(gs_ctx* ctx, const gs_camera* cams, int32_t B, const float* targets, int64_t step);

/* gs_train_graph_launch with the batch's targets in HOST memory (image
 * layout, float32) and the loss read back to host memory: the targets are
 * uploaded on the context's own copy stream into one of two device buffers,
 * so the upload for the next call overlaps this replay (overlap needs
 * page-locked host memory; pageable memory works but copies synchronously).
 * The call first waits until the previous replay has started (has copied
 * its staging area), so that the upload never queues ahead of that copy.
 * The host buffers must stay valid and unchanged until the step has run
 * (gs_sync); *host_loss (may be NULL; page-locked for an asynchronous read)
 * holds the step's loss after gs_sync.
 * Errors: those of gs_train_graph_launch, GS_ENOMEM, GS_ECUDA. */
gs_status gs_train_graph_launch_host(gs_ctx* ctx, const gs_camera* cams, int32_t B, const float* host_targets,
                                     int64_t step, float* host_loss);

/* ---------------------------------------------------------------- serving */

/* Render server: the trained Gaussians stay resident and camera requests of
 * any resolution are batched continuously (the paper's goal is interactive
 * visualisation of the trained model, Sections I and V).  A worker thread
 * forms a batch from the oldest pending requests whenever a slot is free and
 * renders it (projection, binning, forward compositing) on the slot's own
 * context and stream, so batches overlap on the device.  Each result is the
 * same whether rendered alone or in a mix.
 *
 * Memory: at creation every slot reserves, once, the workspaces of its
 * largest batch -- max_batch_views views of max_view_pixels, i.e. per view 72
 * bytes per resident Gaussian (stride), 20 bytes per pixel and 8 bytes per
 * 16x16 tile (max_view_pixels / 128 + 64 tiles) -- and the rest of its share
 * of the budget (memory_budget_bytes / slots, less 1 MiB) as room for tile
 * instances at 26 bytes each (at most 2^30 - 2).  Nothing is allocated or
 * waited for while batches are launched.  A batch is admitted into a slot by
 * that room: each request is charged an instance estimate (1.25 x the most a
 * view of its pixel count has needed so far; for a size not seen yet, two
 * per resident Gaussian plus four per pixel), and a batch takes the oldest
 * pending requests while their estimates fit.  A batch whose instances
 * exceed its estimate is rendered again (its requests go back to the front
 * of the queue; the estimates have learnt the true counts); a request that
 * alone overflows the whole room, or overflows 5 times, completes with
 * GS_ECAPACITY.  A bounded device wait that runs out completes the batch's
 * requests with GS_ETIMEOUT. */
typedef struct gs_server gs_server;

typedef struct {
  int32_t slots;               /* batches in flight, 1..16 (default 2) */
  int32_t max_batch_views;     /* views per batch, 1..64 (default 16) */
  int32_t max_queue;           /* pending requests before GS_EBUSY (default 4096) */
  int32_t max_view_pixels;     /* largest width x height of a request (default 3840 x 2160) */
  int64_t memory_budget_bytes; /* reservation of all slots (default 16 GiB); see above */
  int64_t output_pool_bytes;   /* server-owned output pool; 0 = callers pass outputs */
} gs_serve_cfg;

/* Start a server on `device` for the resident set (device memory owned by
 * the caller, unchanged while the server lives).  cfg may be NULL.
 * Errors: GS_EINVAL (bad cfg, or a budget that leaves a slot room for fewer
 * than 65,536 instances), GS_ENOMEM, GS_ECUDA. */
gs_status gs_serve_create(gs_server** out, int device, const gs_params* resident, const gs_serve_cfg* cfg);

/* Stop the worker, wait for running batches and free the server. */
void gs_serve_destroy(gs_server* srv);

/* Queue one camera.  out_device: device buffer of 3*W*H floats (planar RGB)
 * that receives the image, or NULL to use the server's output pool (then
 * gs_serve_release frees the region).  *ticket identifies the request.
 * Errors: GS_EINVAL (bad camera, W*H above max_view_pixels or more tiles
 * than max_view_pixels / 128 + 64, NULL output without a pool), GS_EBUSY
 * (queue full or output pool full). */
gs_status gs_serve_submit(gs_server* srv, const gs_camera* cam, float* out_device, uint64_t* ticket);

/* Wait up to timeout_us (0 = do not wait, negative = no limit) for a request.  On completion
 * returns GS_OK with *image = its device image and *result = its status;
 * GS_EAGAIN if not done in time; GS_EINVAL for an unknown ticket. */
gs_status gs_serve_poll(gs_server* srv, uint64_t ticket, int64_t timeout_us, const float** image,
                        gs_status* result);

/* Forget a completed request (and free its pool region).  GS_EBUSY if it is
 * still pending or running. */
gs_status gs_serve_release(gs_server* srv, uint64_t ticket);

/* Counters: batches launched (re-renders after a capacity overflow
 * included), requests completed with GS_OK, requests pending. */
gs_status gs_serve_stats(gs_server* srv, int64_t* batches, int64_t* rendered, int64_t* pending);

/* Device timeline of the most recent retired batches (up to 4096 kept):
 * start_end_ms (host, 2 x cap doubles) receives, oldest first, each batch's
 * start and end in milliseconds since the server was created (CUDA events on
 * the slots' streams, so intervals of different slots are comparable and
 * overlap when their batches ran at the same time); *count = pairs written;
 * *retried (may be NULL) = batches rendered again after a capacity overflow.
 * Errors: GS_EINVAL. */
gs_status gs_serve_timeline(gs_server* srv, double* start_end_ms, int32_t cap, int32_t* count, int64_t* retried);

/* ---------------------------------------------------------------- inspection */

/* Intermediate buffers of the last batch (device pointers owned by the
 * context, valid until the next call that rewrites them).  REC0..REC2 are
 * interleaved: entry i of each is at byte offset 48 i from its pointer
 * (one 48-byte record of three float4 per (view, Gaussian)). */
typedef enum {
  GS_BUF_REC0 = 0,   /* float4 [B][N]: mu_x, mu_y, cA, cB with cA = -A log2(e) / 2,
                        cB = -B log2(e) for the conic (A, B, C) */
  GS_BUF_REC1 = 1,   /* float4 [B][N]: cC = -C log2(e) / 2, opacity, red, green */
  GS_BUF_REC2 = 2,   /* float4 [B][N]: blue, hx, hy (half-extents of the box around
                        the alpha >= 1/255 ellipse), depth */
  GS_BUF_KEYS = 3,   /* uint32 [I]: bin of each sorted instance */
  GS_BUF_VALS = 4,   /* uint32 [I]: sorted Gaussian indices */
  GS_BUF_RANGES = 5, /* uint32 [bins][2]: [start, end) per bin */
  GS_BUF_TFINAL = 6, /* float [pixels]: transmittance after the last contributor */
  GS_BUF_NLAST = 7,  /* uint32 [pixels]: 1 + list position of the last contributor */
  GS_BUF_G2D = 8,    /* float [B][N][8] records dL/d(mu_x, mu_y, A, B), dL/d(C, opacity), 0, 0,
                        then [B][N][4] records dL/d(r, g, b), 0 */
  GS_BUF_REC3 = 9,   /* int4 [B][N]: radius (0: the radius' rect misses the
                        view), tiles that receive the Gaussian (0: none), and
                        their rect x0 | x1 << 16, y0 | y1 << 16 (half-open): the
                        radius' rect cut to the tiles the alpha box reaches */
  GS_BUF_SORT_CTRL = 10, /* uint32 [npass + 1]: control word of each pass of the
                        instances' sort by bin; bit 1 set = pass skipped (its
                        digit is the same for every key of each view), bit 0 =
                        source buffer */
  GS_BUF_VISMASK = 11, /* uint64 [N]: bit v = the Gaussian's radius rect meets view
                        v of the last projected batch */
  GS_BUF_DEPTH_CTRL = 12 /* uint32 [5]: control words of the 4 passes of the visible
                        Gaussians' sort by depth bits, as GS_BUF_SORT_CTRL */
} gs_buffer;

/* *ptr = device pointer of the buffer, *count = number of elements (of the
 * type listed above) that are valid.  Errors: GS_EINVAL, GS_ESTATE. */
gs_status gs_get_buffer(gs_ctx* ctx, int32_t which, void** ptr, int64_t* count);

/* Sizes of the last batch: instances I, tile bins, pixels (per channel).
 * Synchronises the stream to read the device-side instance count. */
gs_status gs_get_counts(gs_ctx* ctx, int64_t* instances, int64_t* bins, int64_t* pixels);

/* Work counters of the last forward pass, for the compositing roofline (not
 * part of the training step; one extra pass over the lists, then a stream
 * synchronisation).  *entries = sum over pixels of the list entries up to and
 * including the pixel's last contributor (what the backward walks; a lower
 * bound of what the forward walks); *contributing = the pairs among them with
 * power <= 0 and alpha >= 1/255 (the pairs that change the pixel; the
 * compositing rule of step 3), decided with the compositing kernels' own FP32
 * instruction sequence.  Errors: GS_EINVAL, GS_ESTATE (no forward pass, or
 * inside a graph capture), GS_ENOMEM, GS_ECUDA. */
gs_status gs_pair_stats(gs_ctx* ctx, int64_t* entries, int64_t* contributing);

/* ---------------------------------------------------------------- profiling */

/* Per-kernel accounting: every launch the library makes is counted; while
 * profiling is enabled, CUDA events on the context's stream bracket each
 * launch and their elapsed time is summed per kernel. */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms; /* summed event time (profiling enabled only) */
} gs_kernel_stat;

/* Turn event timing on (enable != 0) or off.  Errors: GS_EINVAL. */
gs_status gs_profile_enable(gs_ctx* ctx, int32_t enable);

/* Copy up to `cap` kernel statistics into out (host array) and set *count to
 * the number of kernels seen.  Synchronises the stream when timings are
 * pending.  Errors: GS_EINVAL, GS_ECUDA. */
gs_status gs_profile_read(gs_ctx* ctx, gs_kernel_stat* out, int32_t cap, int32_t* count);

/* Zero the launch counts and timings (synchronises pending timings away). */
gs_status gs_profile_reset(gs_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* GS_H */
