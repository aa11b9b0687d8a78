/*
 * convex_splat.h -- C ABI of the GB300 (sm_103a) differentiable tile rasterizer for 3D smooth
 * convexes (3D Convex Splatting, arXiv 2411.14974).
 *
 * The library renders a set of N smooth convexes, each the convex hull of K free 3D points
 * (Sec. 3.2, "point-based 3D convex shape representation"), into one or more pinhole views, and
 * computes the gradient of a scalar loss with respect to the points, delta, sigma, opacity and
 * spherical-harmonic colour (Sec. 3.3, "We optimize the position of each point set in 3D, delta
 * and sigma parameters, the opacity o, and the spherical harmonic color coefficients").
 *
 * Per view and convex: the K points are projected (Eq. 4, with the perspective divide), their
 * 2D convex hull is found by Graham scan with exact orientation predicates (Sec. 3.2), the hull
 * edges become lines L_t(q) = n_t . q + c_t with outward unit normals (2D form of Eq. 1), and
 * delta and sigma are multiplied by d^dist_power, d the camera distance (Sec. 3.2 last paragraph,
 * supplementary Eq. S1/S2).  Convexes are binned into 16x16 pixel tiles and sorted by increasing
 * camera distance to their centre (Sec. 3.2), and every pixel q composites front to back
 * (Eq. 5) with
 *     phi(q)   = log sum_t exp(d delta L_t(q))           (Eq. 2 / S1)
 *     I(q)     = Sigmoid(-d sigma phi(q))                (Eq. 3 / S2)
 *     alpha    = min(alpha_max, o I(q)),  skipped if alpha < tau
 *     C(q)    += T alpha c,  T *= (1 - alpha),  stop once T < t_min (after accumulating)
 *     C(q)    += T bg  at the end
 * where c = max(0, sum_lm sh_lm Y_lm(dir) + 0.5) is the view-dependent colour (Sec. 3.2, real
 * SH up to degree 3, dir from the camera centre to the convex centre).
 *
 * Conventions for every entry point:
 *   - Pointers named "device" are CUDA device memory on the context's device, owned by the
 *     caller; the library never frees them and only reads inputs / writes outputs.
 *   - Pointers named "host" are ordinary (preferably pinned) host memory owned by the caller.
 *   - Layouts are dense, C order, float32 unless stated:
 *       points  [N][K][3], delta/sigma/opacity [N], sh [N][(D+1)^2][3]   (D = sh_degree)
 *       image   [V][3][H][W] (channel planes), t_final [V][H][W]
 *   - Every call returns a cs_status and never aborts, throws or traps.  On failure
 *     cs_last_error() (thread-local) describes the cause.  Asynchronous device errors are
 *     reported by the next call that synchronises.
 *   - The stream argument is a cudaStream_t (0 = legacy default stream).  Work is enqueued on it;
 *     cs_forward waits once on the host, for the preprocess's totals (the tile-pair count that sizes
 *     the pair buffers, and the range of the depth keys); work it has already queued keeps running.
 */
#ifndef CONVEX_SPLAT_H
#define CONVEX_SPLAT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    CS_OK = 0,
    CS_ERR_ARG = 1,      /* invalid argument (null pointer, size, unsupported setting) */
    CS_ERR_CUDA = 2,     /* a CUDA runtime call failed */
    CS_ERR_NOMEM = 3,    /* device or host allocation failed */
    CS_ERR_BUDGET = 4,   /* a serving request does not fit the memory budget */
    CS_ERR_TIMEOUT = 5,  /* a bounded wait ran out */
    CS_ERR_DEVICE = 6,   /* checked builds only: a kernel's index test failed (status word) */
    CS_ERR_STATE = 7     /* object used in the wrong state (e.g. released, unknown id) */
} cs_status;

/* Pinhole camera (Eq. 4).  World -> camera rotation R (row major) and translation t, OpenCV axes
   (x right, y down, z forward).  Pixel (i, j) is sampled at (i + 0.5, j + 0.5); a point maps to
   (fx x/z + cx, fy y/z + cy).  Convexes with any point at z < z_near are not drawn. */
typedef struct {
    int32_t width, height;
    float fx, fy, cx, cy;
    float R[9];
    float t[3];
    float z_near;
} cs_camera;

/* Compositing constants.  The paper's Eq. 5 has none; these follow the 3DGS tile rasterizer the
   paper builds on (Sec. 3.2).  cs_default_settings(): tau = 1/255, alpha_max = 0.99,
   t_min = 1e-4, bg = 0, dist_mode = 0, dist_power = 1, tile_test = 0, tile_split = 0. */
typedef struct {
    float tau;          /* pairs with alpha < tau add nothing; 0 <= tau < 1 */
    float alpha_max;    /* alpha = min(alpha_max, o I); 0 < alpha_max <= 1 */
    float t_min;        /* compositing stops once T < t_min (after accumulating); 0 <= t_min < 1 */
    float bg[3];        /* background colour added with the final transmittance */
    int32_t dist_mode;  /* d = |R c + t| (0) or the camera z of c (1); c = mean of the K points */
    float dist_power;   /* delta, sigma scaled by d^p, p in {0, 0.5, 1, 2} (supp. Sec. C ablation) */
    int32_t tile_test;  /* 0: a convex covers every tile of its conservative rectangle; 1: only the
                           tiles an exact separating-axis test against its offset hull keeps (fewer
                           pairs, more work per convex; see the tile-range notes of cs_forward) */
    int32_t tile_split; /* 0: one CTA blends each tile.  N in 256..2^24: a tile with more than N
                           pairs is blended as chunks of N pairs by separate CTAs, merged in depth
                           order by C = C_a + T_a C_b, T = T_a T_b, with the chunk in which a
                           pixel's walk stops (T < t_min) walked again from T_a, so the image is
                           that of the unsplit walk; the backward runs per chunk from the merged
                           state.  Costs one more host synchronisation per forward and 5 KB of
                           state per chunk of a heavy tile.  Ignored by cs_forward_static. */
} cs_settings;

/* How delta, sigma and opacity are given (Sec. 3.3 optimises them through activations). */
typedef enum {
    CS_ACT_NONE = 0,         /* activated values: delta, sigma > 0, opacity in (0, 1] */
    CS_ACT_EXP_SIGMOID = 1   /* training parameters: delta = exp(x), sigma = exp(x), opacity = sigmoid(x)
                                of the stored x, applied inside the forward; the backward then returns
                                gradients with respect to the stored x.  exp is one fixed binary32
                                definition (Cody-Waite reduction with ln 2 split into a 16-bit head
                                and a tail, degree-7 Taylor polynomial by Horner, times 2^k; 0 below
                                2^-126, +inf above the binary32 range), sigmoid(x) = 1/(1 + exp(-x)) */
} cs_activation;

/* Element type of a scene's parameter arrays.  The 16-bit formats are the paper's "light" model
   storage (Sec. 4.2, supplement Sec. A: weights stored in 16-bit precision); every value is
   widened to binary32 on load and all arithmetic is binary32, so a 16-bit scene renders exactly
   like the binary32 scene holding the same (widened) values.  Gradients are always float32. */
typedef enum {
    CS_STORE_F32 = 0,
    CS_STORE_F16 = 1,   /* IEEE binary16 */
    CS_STORE_BF16 = 2   /* bfloat16 */
} cs_storage;

/* A scene: device pointers to N convexes with K points each (3 <= K <= 8) and SH degree D (0..3),
   every array of the element type `storage`: points [N][K][3], delta [N], sigma [N], opacity [N],
   sh [N][(D+1)^2][3].  Convexes whose (activated) delta/sigma are non-finite or non-positive are
   not drawn. */
typedef struct {
    const void *points;
    const void *delta;
    const void *sigma;
    const void *opacity;
    const void *sh;
    int64_t n;
    int32_t k;
    int32_t sh_degree;
    int32_t activation;   /* cs_activation */
    int32_t storage;      /* cs_storage */
} cs_scene;

typedef struct cs_context cs_context;      /* per-device library state: stream-ordered memory pool */
typedef struct cs_fwd_state cs_fwd_state;  /* what a forward keeps for its backward */

/* Fill *s with the defaults listed above. */
void cs_default_settings(cs_settings *s);

/* Thread-local description of the last failure on this thread ("" if none). */
const char *cs_last_error(void);

/* Create a context on CUDA device `device`.  The context owns a stream-ordered memory pool for
   the transient buffers of every call made with it, and the forward's readback slot, so calls on
   one context must not overlap: use one context per host thread (the serving loop makes its own).
   Returns CS_ERR_CUDA if the device cannot be used (no GPU, wrong architecture). */
cs_status cs_context_create(int32_t device, cs_context **out);
void cs_context_destroy(cs_context *ctx);

/* Forward render (Sec. 3.2, Eq. 4, 5, S1, S2) of `scene` into n_views views of equal size.
   cams:    host array [n_views]; all views must have the same width and height.
   image:   device [n_views][3][H][W], written.
   t_final: device [n_views][H][W] final transmittance, written; may be NULL.  Neither image nor
            t_final is read again by cs_backward (the state keeps its own copy).
   state_out: if not NULL, receives a new state holding what cs_backward needs (the sorted
            tile-pair lists, per-convex screen records, per-pixel T_final and last contributor);
            release it with cs_state_release.  The scene buffers must stay alive and unchanged
            until the backward has run.
   Errors: CS_ERR_ARG for bad sizes/settings, CS_ERR_NOMEM, CS_ERR_CUDA. */
cs_status cs_forward(cs_context *ctx, const cs_scene *scene, const cs_camera *cams, int32_t n_views,
                     const cs_settings *settings, float *image, float *t_final, cs_fwd_state **state_out,
                     void *stream);

/* Backward of cs_forward: given dL/dimage (device, same layout as image) accumulate (+=) the
   gradient into the caller's device buffers dpoints [N][K][3], ddelta [N], dsigma [N],
   dopacity [N], dsh [N][(D+1)^2][3] (any may be NULL to skip it; none may alias).  Reverse-order
   compositing recomputes the transmittance from T_final (no per-pair storage); per-convex
   gradients are reduced within each warp before global atomics.  Kinks take the one-sided value
   0: clamped alpha, colour clamped at 0, skipped pairs. */
cs_status cs_backward(cs_context *ctx, const cs_fwd_state *state, const float *dL_dimage, float *dpoints,
                      float *ddelta, float *dsigma, float *dopacity, float *dsh, void *stream);

/* cs_backward, except that the gradients are written instead of added to the buffers' contents:
   the buffers need not be cleared first (with several views the call clears them, then adds the
   views' contributions).  With one view the preprocess backward then reads no old gradient, 264
   of its 988 bytes per convex at K = 6 and SH degree 3.  Same arguments and errors. */
cs_status cs_backward_write(cs_context *ctx, const cs_fwd_state *state, const float *dL_dimage, float *dpoints,
                            float *ddelta, float *dsigma, float *dopacity, float *dsh, void *stream);

/* Release a state (its device buffers return to the context's pool on the state's stream). */
void cs_state_release(cs_fwd_state *state);

/* Internal arrays of a forward state, copied to host memory for inspection and parity checks.
   which: see cs_array.  host_dst may be NULL to query the size.  Synchronous. */
typedef enum {
    CS_ARR_RECORDS = 0,      /* float [R][32]: per (view, convex) screen record: anchor vertex (x, y),
                                d^p sigma, opacity, rgb, packed hull (T | index_i << (4 + 3 i)), then
                                per hull line t < 8 (A, B, C) = log2(e) d^p delta (n_x, n_y,
                                n . (anchor - v_t)), i.e. lines relative to the anchor */
    CS_ARR_DEPTH_KEYS = 1,   /* uint32 [R]: binary32 bits of the camera distance; 0xffffffff if not drawn */
    CS_ARR_RECTS = 2,        /* uint32 [R][2]: tile range (tx0 | tx1 << 16, ty0 | ty1 << 16) */
    CS_ARR_COUNTS = 3,       /* uint32 [R]: number of tiles the convex covers (the whole range, or the
                                tiles the exact tile test keeps); 0 if not drawn */
    CS_ARR_PAIR_KEYS = 4,    /* uint32 [P]: view << b | tile index within the view, b = bits of the largest
                                view's tile count (one view: the tile index); the device copy also
                                holds an 8-bit block mask above these bits, which the copy removes */
    CS_ARR_PAIR_VALUES = 5,  /* uint32 [P]: record index (view * N + convex) of each sorted pair */
    CS_ARR_TILE_RANGES = 6,  /* uint32 [tiles][2]: [start, end) of each tile in the pair list; tiles of
                                all views in view order, row major within a view */
    CS_ARR_N_LAST = 7,       /* uint32 [V][H][W]: 1 + pair index of the last contributor, 0 if none */
    CS_ARR_HULLS = 8,        /* uint32 [R]: hull size T in bits 0-3, vertex i in bits 4+3i.. */
    CS_ARR_TILE_ORDER = 9    /* uint32 [tiles]: the order in which the blend kernels take the tiles, a
                                permutation of the tile indices by decreasing floor(log2(pairs + 1))
                                (any order within a class); empty (0 bytes) when the blends run in
                                chunks (tile_split) or per view (serving) */
} cs_array;
cs_status cs_state_copy(const cs_fwd_state *state, int32_t which, void *host_dst, size_t capacity,
                        size_t *bytes_out);

/* Numbers of records R (= n_views * N), sorted pairs P and tiles of a forward state. */
cs_status cs_state_sizes(const cs_fwd_state *state, int64_t *records, int64_t *pairs, int64_t *tiles);

/* One forward (and, if dL_dimage_host is not NULL, backward) with every buffer in HOST memory
   (preferably pinned): the scene arrays are copied to the device and rendered; the image,
   dL_dimage and, with one view, the gradients are written and read in place by the kernels when
   the device can reach the host buffers (pinned or registered memory, or any memory on a host
   whose page tables the GPU uses, as a Grace host over NVLink-C2C), so that the gradients stream
   out while they are computed; otherwise they go through device buffers and copies.  Same
   layouts as cs_forward / cs_backward; scene_host holds host pointers.  The gradients are written
   (not accumulated); any gradient pointer may be NULL.  Device buffers come from the context's
   pool; the call synchronises. */
cs_status cs_step_host(cs_context *ctx, const cs_scene *scene_host, const cs_camera *cams, int32_t n_views,
                       const cs_settings *settings, const float *dL_dimage_host, float *image_host,
                       float *dpoints_host, float *ddelta_host, float *dsigma_host, float *dopacity_host,
                       float *dsh_host, void *stream);

/* Pipelined host-buffer steps (no counterpart in the paper).  cs_step_host_submit enqueues the work
   of cs_step_host for one view and returns a ticket without waiting for any of it.  The context
   keeps three slots of device buffers (scene, dL_dimage, image, gradients), three streams and one
   worker thread of its own: the calling thread copies a step's scene and dL_dimage into its slot
   on the upload stream and queues the step; the worker thread enqueues the step's forward and
   backward on the compute stream (it, not the caller, waits there for the forward's pair count)
   and the copies of its image and gradients on the download stream.  So later steps' inputs
   arrive and earlier steps' outputs leave over the host link while the GPU computes.  A submit
   waits only when the step three tickets back has not yet been enqueued by the worker (its slot
   is reused).  The host buffers should be pinned (or registered): a copy to or from pageable
   memory makes the call wait for it.  The gradients are written, not accumulated; any gradient
   pointer may be NULL, and dL_dimage NULL runs the forward only.  Until cs_step_host_wait(ticket)
   returns, the step's host arrays must not change and its outputs must not be read, and the
   context must be given no call other than cs_step_host_submit and cs_step_host_wait.  Steps
   complete in submission order: waiting for a ticket waits for every earlier step of the context
   too.  The slots (cudaMalloc'd, grown to the largest step submitted), the streams and the thread
   are kept until cs_context_destroy, which lets the thread enqueue the steps still queued and
   waits for them.  Errors: the submit reports argument errors (CS_ERR_ARG, also for a ticket not
   yet submitted) and failures of the upload (CS_ERR_CUDA); a failure of a queued step's forward,
   backward or download (the codes of cs_forward and cs_backward_write) is returned, with its
   message, by the next cs_step_host_wait, once. */
cs_status cs_step_host_submit(cs_context *ctx, const cs_scene *scene_host, const cs_camera *cam,
                              const cs_settings *settings, const float *dL_dimage_host, float *image_host,
                              float *dpoints_host, float *ddelta_host, float *dsigma_host, float *dopacity_host,
                              float *dsh_host, uint64_t *ticket);
cs_status cs_step_host_wait(cs_context *ctx, uint64_t ticket);

/* ---- forward that allocates nothing (no counterpart in the paper) ---------------------------
   For callers that cannot allocate device memory at the point where they render: an engine that
   owns every byte of device memory through its own arena (a hidden cudaMalloc would escape its
   accounting), a real-time loop that must not enter the driver's allocator (it can block or
   synchronise), or a plugin that may only allocate while it is being set up.
   cs_forward_static renders ONE view (the same computation as cs_forward with n_views = 1) and
   takes every transient buffer from a fixed device array of CS_STATIC_SCRATCH_BYTES declared at
   file scope in the library; it calls no cudaMalloc, cudaFree or other allocating routine.
   scene: device pointers as for cs_forward.  image [3][H][W] and t_final [H][W]: device, written,
   both required.  Limits: n <= CS_STATIC_MAX_CONVEXES, width * height <= CS_STATIC_MAX_PIXELS
   (1920x1080 fits), tile pairs <= CS_STATIC_MAX_PAIRS; beyond a limit the call returns
   CS_ERR_BUDGET with a message and leaves image and t_final untouched.
   Every GPU that loads the library holds the array until the process exits.  All calls share it
   and it keeps the last call's contents (each call clears on its stream what must start at zero),
   so calls that overlap on the GPU race: issue them on one stream, one after the other.  The first
   call on a device looks up the array's device address with that device current: make that first
   call before any stream capture.  The call synchronises its stream once (to read the number of
   tile pairs) and keeps no state for a backward. */
#define CS_STATIC_SCRATCH_BYTES (32u << 20)
#define CS_STATIC_MAX_CONVEXES 65536
#define CS_STATIC_MAX_PIXELS (1 << 21)
#define CS_STATIC_MAX_PAIRS (1 << 19)
cs_status cs_forward_static(const cs_scene *scene, const cs_camera *cam, const cs_settings *settings, float *image,
                            float *t_final, void *stream);

/* ---- training step around the renderer (Sec. 3.3) --------------------------------------------
   With scene.activation = CS_ACT_EXP_SIGMOID the forward/backward above work on the training
   parameters directly; these two calls add the loss and the optimiser, all on the device. */

/* Photometric loss of Sec. 3.3 (Eq. 6 without the mask term, lambda = 0.2 in the paper):
     L = (1 - lambda) mean|image - target| + lambda (1 - mean SSIM(image, target))
   over n_views x 3 x height x width elements (layout [V][3][H][W], float32, device).  SSIM per
   Wang et al. (2004): 11 x 11 Gaussian window of standard deviation 1.5, C1 = 0.01^2,
   C2 = 0.03^2, statistics per channel plane with zero padding outside the image.
   loss_out (device, one float) receives L when not NULL.  dL_dimage (device, same layout as
   image) is overwritten with dL/dimage when not NULL; the L1 subgradient at image == target is 0.
   Transient buffers (3 floats per element) come from ctx's pool.  0 <= lambda <= 1; at most
   21845 views per call.  Errors: CS_ERR_ARG for bad sizes or NULL inputs, CS_ERR_CUDA. */
cs_status cs_loss_l1_dssim(cs_context *ctx, const float *image, const float *target, int32_t n_views,
                           int32_t height, int32_t width, float lambda, float *loss_out, float *dL_dimage,
                           void *stream);

/* One Adam update (Kingma and Ba 2015, Algorithm 1) of up to CS_ADAM_MAX_GROUPS parameter arrays
   in one launch, in binary32 per element:
     m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;
     p -= lr (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps),  t = step >= 1.
   Every pointer of a group is a caller-owned device float array of n elements (m and v start at
   0 and persist between steps).  grad_abs_sum, when not NULL, receives += |g| per element (the
   per-convex statistic of the split criterion when the group is sigma).  zero_grad != 0 sets the
   gradient to 0 after use, ready for the next backward to accumulate into.  Groups with n = 0 are
   skipped.  Errors: CS_ERR_ARG (NULL buffers, n < 0, step < 1, beta outside [0, 1)), CS_ERR_CUDA. */
#define CS_ADAM_MAX_GROUPS 16
typedef struct {
    float *param;
    float *grad;
    float *m;
    float *v;
    float *grad_abs_sum;  /* optional */
    int64_t n;
    float lr;
} cs_adam_group;

typedef struct {
    float beta1;      /* 0.9 */
    float beta2;      /* 0.999 */
    float eps;        /* 1e-15 */
    int32_t zero_grad;
} cs_adam_settings;

cs_status cs_adam_step(cs_context *ctx, const cs_adam_group *groups, int32_t n_groups,
                       const cs_adam_settings *settings, int64_t step, void *stream);

/* Adaptive refinement (Sec. 3.3, supplement Sec. A): split and prune a set of raw training
   parameters (points, log delta, log sigma, logit opacity, SH; the CS_ACT_EXP_SIGMOID convention)
   together with their Adam moments.  Per convex, decided in binary32:
     prune  when sigmoid(opacity) < prune_opacity, when its size (largest distance from its centre,
            the mean of its points, to one of its points) exceeds prune_size, or when a point is
            not finite;
     split  otherwise when sigma_grad_abs / window_steps > split_threshold (the mean |dL/dsigma|
            since the last refinement, as accumulated by cs_adam_step);
     keep   otherwise.
   Output, in input order: a kept convex once (with its moments), a split convex as K children
   (child j: points p_j + split_scale (p_k - c), same delta and SH, sigma x split_sigma_scale,
   opacity x split_opacity_scale, i.e. raw sigma + ln(scale) and raw opacity ln(o'/(1 - o')) with
   the binary32 ln of the tile range; moments 0), a pruned one not at all.
   out_* must not alias the inputs and hold `capacity` convexes.  *n_out (host) receives the
   output count; the call synchronises the stream once to read it.  If it exceeds capacity the
   call returns CS_ERR_BUDGET with *n_out set and writes no output (decisions are written).
   adam_m/adam_v/out_m/out_v are all given or all NULL.  decisions (device int32 [n], 0 keep,
   1 split, 2 prune) is optional. */
typedef struct {
    float *points;   /* [N][K][3] */
    float *delta;    /* [N] */
    float *sigma;    /* [N] */
    float *opacity;  /* [N] */
    float *sh;       /* [N][(D+1)^2][3] */
} cs_param_arrays;

typedef struct {
    float split_threshold;      /* 4e-6 (supplement Sec. A) */
    float split_scale;          /* 0.7 (indoor) or 0.6 (outdoor) */
    float split_sigma_scale;    /* > 0; 1.5 */
    float split_opacity_scale;  /* (0, 1]; 0.5 */
    float prune_opacity;        /* 0.03 */
    float prune_size;           /* 0.3 x scene size; +inf disables */
} cs_refine_settings;

cs_status cs_refine(cs_context *ctx, int64_t n, int32_t k, int32_t sh_degree, const cs_param_arrays *params,
                    const cs_param_arrays *adam_m, const cs_param_arrays *adam_v, const float *sigma_grad_abs,
                    int32_t window_steps, const cs_refine_settings *settings, int64_t capacity,
                    cs_param_arrays *out_params, cs_param_arrays *out_m, cs_param_arrays *out_v, int32_t *decisions,
                    int64_t *n_out, void *stream);

/* ---- serving: continuous batching of novel-view requests (no counterpart in the paper) -------
   A server keeps several scenes resident (device buffers owned by the caller, registered with
   cs_server_add_scene) and renders view requests of mixed resolution.  A worker thread admits
   queued requests in arrival order into a batch of at most max_batch views, as long as the
   estimated transient memory of the batch plus what the batches still on the GPU hold (their
   estimates, or the server's memory pool's real usage when that is more) fits the memory
   budget; requests that arrive while earlier batches are on the GPU join the next batch as soon
   as memory frees up.  A batch is preprocessed, binned and sorted as one (the view index lives in
   the tile key), then blended by one persistent launch (batches of at most 32 views; larger ones
   launch one blend per view) that takes the tiles view by view, cheapest view first; each
   request completes as soon as its own view's image is written (the launch raises a flag per
   view in mapped host memory, which the server's finisher thread polls).  Batches alternate
   between two streams, at most one in flight on each, so the preprocess and sorts of one overlap
   the blends of the previous one.  Each view's image is identical to rendering it alone with
   cs_forward.
   Images are written to caller-owned device buffers [3][H][W] that must stay alive until the
   request's completion has been polled.  All calls are thread-safe. */
typedef struct cs_server cs_server;

typedef struct {
    uint64_t id;          /* request id returned by cs_server_submit */
    int32_t status;       /* CS_OK, CS_ERR_BUDGET (larger than the whole budget), CS_ERR_STATE
                             (scene removed while queued), CS_ERR_CUDA */
    int32_t batch_size;   /* views in the batch that rendered it */
    double queue_ms;      /* submit -> batch admitted */
    double latency_ms;    /* submit -> image complete on the device */
} cs_completion;

/* memory_budget_bytes bounds the transient device memory of admitted batches (see above);
   1 <= max_batch <= 1024.  settings apply to every request. */
cs_status cs_server_create(int32_t device, size_t memory_budget_bytes, int32_t max_batch, const cs_settings *settings,
                           cs_server **out);
/* Stops the worker after the queued requests complete, then frees the server. */
void cs_server_destroy(cs_server *srv);
/* on = 1 (the default): the worker admits the next batch while earlier ones are still on the GPU
   (two streams).  on = 0: the worker waits for each batch to finish on the GPU before it admits
   the next, so batches never overlap; with max_batch = 1 that is plain one-view-at-a-time
   rendering, the baseline the serving measurements compare against.  Applies from the next
   batch on. */
cs_status cs_server_set_pipelining(cs_server *srv, int32_t on);
/* Registers a resident scene (device pointers as for cs_forward; the caller keeps them alive and
   unchanged while the scene is registered).  Returns its id in *scene_id. */
cs_status cs_server_add_scene(cs_server *srv, const cs_scene *scene, int32_t *scene_id);
/* Unregisters a scene; its queued requests complete with CS_ERR_STATE, batches already admitted
   finish normally.  Returns once no admitted batch still reads the scene. */
cs_status cs_server_remove_scene(cs_server *srv, int32_t scene_id);
/* Queues a view of scene_id; image: device [3][cam->height][cam->width].  CS_ERR_ARG for a bad
   camera or unknown scene (nothing is queued). */
cs_status cs_server_submit(cs_server *srv, int32_t scene_id, const cs_camera *cam, float *image,
                           uint64_t *request_id);
/* Moves up to max completions into out (oldest first); waits up to wait_ms milliseconds for the
   first one when none is ready (0 = do not wait). */
cs_status cs_server_poll(cs_server *srv, cs_completion *out, int32_t max, int32_t *n_out, int32_t wait_ms);
/* Counters (stats: 7 values): [0] requests completed, [1] batches run, [2] largest batch,
   [3] peak estimated bytes in flight, [4] requests queued now, [5] requests on the GPU now,
   [6] peak bytes the server's memory pool really held for batches (its high-water mark since
   cs_server_create). */
cs_status cs_server_stats(cs_server *srv, uint64_t *stats);

/* ---- instrumentation (no counterpart in the paper) ------------------------------------------ */
typedef enum {
    CS_STAGE_PREPROCESS = 0,      /* per-convex projection, hull, lines, tile range, colour */
    CS_STAGE_DEPTH_SORT = 1,      /* radix sort of the records by depth key */
    CS_STAGE_SCAN_EMIT = 2,       /* tile-count scan, pair-count readback, pair emission */
    CS_STAGE_TILE_SORT = 3,       /* radix sort of the pairs by tile, tile ranges */
    CS_STAGE_BLEND = 4,           /* per-tile forward compositing */
    CS_STAGE_BLEND_BACKWARD = 5,  /* per-tile reverse compositing, per-convex gradient records */
    CS_STAGE_PREPROCESS_BACKWARD = 6, /* chain to points, delta, sigma, opacity, SH */
    CS_STAGE_LOSS = 7,            /* cs_loss_l1_dssim */
    CS_STAGE_OPTIMIZER = 8,       /* cs_adam_step */
    CS_STAGE_COUNT = 9
} cs_stage;

/* When on, every stage of every call on this context is bracketed by CUDA events recorded on the
   stream the stage is launched on. */
cs_status cs_profile_enable(cs_context *ctx, int32_t on);
/* Sum of the event-timed milliseconds and number of timed launches per stage since the last read
   (arrays of CS_STAGE_COUNT); synchronises on the recorded events, then resets the record. */
cs_status cs_profile_read(cs_context *ctx, double *ms, int64_t *launches);
/* Total number of kernels this library has launched in the process (monotonic). */
uint64_t cs_kernel_launch_count(void);

/* Checked builds (no counterpart in the paper).  The library built with CS_CHECKED=1 tests, in
   its kernels, every index that an inconsistent upstream value could send outside its buffer (a
   tile's pair range, a pair's record index, a record's hull count, an emitted pair slot, a tile
   index, a radix-sort destination); a failed test skips or clamps that access and sets a bit of a
   device status word, never traps.  cs_forward, cs_backward and cs_forward_static then synchronise
   their stream, read and clear the words and return CS_ERR_DEVICE, naming the bits.  Every
   transient buffer is handed out filled with 0xff bytes (NaN as float), so that a read before a
   write changes the results.  The status words are per process and device: concurrent calls share
   them.  Production builds compile all of this out and never return CS_ERR_DEVICE.
   cs_debug_set_pair_value overwrites entry `index` of a forward state's sorted pair values (the
   record each tile pair refers to), so that a test can hand the backward an inconsistent pair list
   for the checks to catch; production builds return CS_ERR_STATE.  Synchronous. */
cs_status cs_debug_set_pair_value(cs_fwd_state *state, int64_t index, uint32_t value);

/* Measured issue rates of the two arithmetic pipes the blend kernels load, on `device`:
   out[0] = ex2.approx results per clock per SM (the transcendental unit), out[1] = FP32 fused
   multiply-adds per clock per SM, out[2] = the SM clock during the measurement (MHz), out[3] =
   the number of SMs.  Each is the median over SMs of results over the cycles (clock64) the SM
   spent on a launch of 8 independent dependency chains per thread; about a millisecond of GPU
   time, synchronous, two small cudaMalloc'd buffers.  Errors: CS_ERR_ARG, CS_ERR_CUDA. */
cs_status cs_measure_alu_rates(int32_t device, double *out);

/* Work actually done by the two blend kernels of a forward state, counted by instrumented
   variants of the kernels (the state's pair lists are re-blended; outputs are unchanged).
   counts[0..5] forward, counts[6..11] backward: pairs visited, hull lines of the visited pairs,
   pairs past the line pre-test, hull lines of those, pairs that contribute (alpha >= tau),
   pixels.  dL_dimage may be NULL (forward counts only). */
cs_status cs_work_counts(cs_context *ctx, const cs_fwd_state *state, const float *dL_dimage, uint64_t *counts,
                         void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CONVEX_SPLAT_H */
