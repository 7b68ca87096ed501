/*
 * ludvig.h -- C ABI of libludvig, a GB300 (sm_103a) implementation of the
 * uplifting and graph-diffusion hot path of LUDVIG (Marrie et al., "LUDVIG:
 * Learning-free Uplifting of 2D Visual features to Gaussian Splatting
 * scenes", arXiv 2410.14462).
 *
 * Conventions shared by every entry point
 *  - Pointers documented as "device" are CUDA device pointers owned by the
 *    caller; the library never frees them.  "host" pointers are ordinary
 *    host memory.  Arrays are dense, row-major, without padding.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *    stream).  Work is enqueued asynchronously on it; argument errors are
 *    reported synchronously before anything is enqueued.  A call returns
 *    LUDVIG_ERR_CUDA if a CUDA runtime call fails; the message is then in
 *    ludvig_last_error().
 *  - The uplift entry points (ludvig_uplift, ludvig_uplift_accumulate,
 *    ludvig_uplift_fp8) do not wait on the host: workspace capacities are
 *    checked on the device and kernel-side failures (an expired bounded
 *    wait) go to the scene's device status word.  ludvig_sync(scene) waits
 *    for the scene's last such call, completes it and returns that status;
 *    the results are final once it returns LUDVIG_OK.  The next call on the
 *    same scene does the same first (so calls on one scene never overlap),
 *    but only ludvig_sync reports the status.  Inputs and outputs of a call
 *    must stay allocated until then.
 *  - Outputs are written only when the call returns LUDVIG_OK.
 *  - A scene (and a graph) may be used by one stream at a time: calls on the
 *    same scene from different streams must be ordered by the caller.
 *    Calls on different scenes and graphs may come from several host
 *    threads at once (the last-error message is per thread).
 *  - The library keeps a per-scene device workspace that grows on demand
 *    (cudaMalloc) and is reused; the first call at a new size allocates (and
 *    synchronises the device, so a growing call waits on the host).
 *    ludvig_uplift_batch lends pooled per-slot workspaces to its jobs
 *    instead, so resident scenes need not each hold one.
 *
 * Geometry conventions (the paper fixes none; these are the 3D Gaussian
 * Splatting rasteriser's, which the paper uses, Sec. 5):
 *  - camera: world point X maps to x = R X + t (OpenCV axes: x right, y down,
 *    z forward) and to pixel coordinates (fx x/z + cx, fy y/z + cy); pixel
 *    (u,v) is sampled at its centre (u+0.5, v+0.5).
 *  - Gaussian i: mean mu_i, covariance Sigma_i = R(q_i) diag(s_i)^2 R(q_i)^T
 *    with q_i = (w,x,y,z) normalised inside the library, s_i the per-axis
 *    standard deviations (given as logarithms, as a trained scene stores
 *    them, or linear: ludvig_scene_opts), opacity o_i in (0,1) (post-sigmoid).
 *  - 2D footprint: EWA covariance J R Sigma R^T J^T + 0.3 I (Jacobian taken at
 *    the mean with x/z, y/z clamped to 1.3 x the half field of view), near
 *    plane z > 0.2, radius ceil(3 sqrt(lambda_max)), 16x16 pixel tiles.
 *  - weights (Sec. 3.1, Eq. 1): along each pixel's depth-ordered list
 *    (ties: lower index first) alpha = min(0.99, o * exp(-0.5 d^T C d)); a
 *    Gaussian with alpha < 1/255 is skipped; the walk stops before the
 *    Gaussian that would take the transmittance below 1e-4;
 *    w = alpha * T.
 */
#ifndef LUDVIG_H
#define LUDVIG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LUDVIG_ABI_VERSION 11

typedef enum {
    LUDVIG_OK = 0,
    LUDVIG_ERR_ARG = 1,          /* invalid argument (nothing enqueued) */
    LUDVIG_ERR_OOM = 2,          /* device allocation failed */
    LUDVIG_ERR_CUDA = 3,         /* a CUDA runtime call failed */
    LUDVIG_ERR_TIMEOUT = 4,      /* a bounded wait expired */
    LUDVIG_ERR_INTERNAL = 5,     /* a device-side consistency check failed */
    LUDVIG_ERR_UNSUPPORTED = 6   /* valid request this build does not implement */
} ludvig_status;

typedef enum {
    LUDVIG_F32 = 0,              /* float32 features.  4 < d < 32, or 32 <= d <= 512 with
                                    d % 8 == 0: tensor-core aggregation with features and weights
                                    split into two bfloat16 terms each (float32-level accuracy);
                                    d <= 4: the same weight terms summed in the compositing pass;
                                    otherwise, or with LUDVIG_OPT_F32_TENSOR_CORES = 0, CUDA-core
                                    FFMA */
    LUDVIG_BF16 = 1              /* bfloat16 features.  4 < d < 32, or 32 <= d <= 512 with
                                    d % 8 == 0: tensor-core aggregation with bfloat16 weights;
                                    d <= 4: bfloat16 weights summed in the compositing pass;
                                    otherwise CUDA cores with float32 weights */
} ludvig_dtype;

/* Process-wide options (ludvig_set_option / ludvig_get_option). */
typedef enum {
    LUDVIG_OPT_F32_TENSOR_CORES = 0,  /* 1 (default): float32 features use the split-bfloat16
                                         tensor-core kernel where it applies; 0: CUDA-core FFMA */
    LUDVIG_OPT_COUNT_NORMALISE = 1,   /* 0 (default): the uplift divides by sum_{v,p} w_i (Eq. 3).
                                         1: GaussianEditor's normaliser (appendix, comparison
                                         with GaussianEditor): the number of (view, pixel) pairs
                                         with w_i > 0; beta/den then hold those counts */
    LUDVIG_OPT_FAULT_ALLOC = 2,       /* host-side fault injection for tests: k > 0 makes the k-th
                                         workspace allocation from now fail once with
                                         LUDVIG_ERR_OOM (nothing is allocated); 0 disarms */
    LUDVIG_OPT_FAULT_LAUNCH = 3,      /* k > 0: the k-th checked kernel launch from now reports
                                         LUDVIG_ERR_CUDA once (the kernel itself was queued and
                                         runs normally); 0 disarms.  The failed call's outputs
                                         are undefined; a later call starts afresh */
    LUDVIG_OPT_AGG_CONFIG = 4,        /* shared-memory layout of the float32 tensor-core
                                         aggregation: 0 = seven feature stages, four epilogue
                                         warps; 1 = five stages, eight epilogue warps.  Results
                                         are the same to rounding; only the speed differs */
    LUDVIG_OPT_GROUP_MB = 5,          /* views per group of the pipeline: up to 128, with their
                                         per-view Gaussian scratch (about 120 bytes per view
                                         and Gaussian) within this many MiB (default 2048,
                                         range 1..65536; a group holds at least one view).  Larger groups take fewer launches
                                         and more workspace; results are the same to rounding */
    LUDVIG_OPT_BATCH_TUNE = 6,        /* 1 (default): ludvig_uplift_batch picks the group size
                                         of each class of jobs by timing candidates on the
                                         class's own jobs the first time it meets the class
                                         (see ludvig_uplift_batch); 0: LUDVIG_OPT_GROUP_MB */
    LUDVIG_OPT_BATCH_PACK = 7,        /* 1 (default): ludvig_uplift_batch packs the views of
                                         tensor-core jobs into shared groups; 0: every job
                                         runs as its own ludvig_uplift call (the unpacked
                                         form, kept for comparison) */
    LUDVIG_OPT_AGG_SMS = 8            /* 0 (default): the tensor-core aggregation runs one
                                         persistent CTA on every SM; k > 0: on at most k SMs,
                                         leaving the others to the next group's front end on
                                         its own stream.  Results are the same to rounding */
} ludvig_option;

/* Sets an option; LUDVIG_ERR_ARG for an unknown option. */
ludvig_status ludvig_set_option(int32_t option, int64_t value);

/* Current value of an option, or -1 for an unknown option. */
int64_t ludvig_get_option(int32_t option);

/* Pinhole camera, host memory.  R: row-major world->camera rotation. */
typedef struct {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
} ludvig_camera;

typedef struct ludvig_scene* ludvig_scene_t;
typedef struct ludvig_graph* ludvig_graph_t;

/* ABI version of the loaded library (LUDVIG_ABI_VERSION it was built with). */
int32_t ludvig_abi_version(void);

/* Thread-local message describing the last failed call on this thread. */
const char* ludvig_last_error(void);

/* Options of ludvig_scene_create (NULL: all zero). */
typedef struct {
    int32_t scales_are_linear;   /* 0: scales are log standard deviations (exponentiated with
                                    float32 expf); 1: linear standard deviations (> 0), e.g.
                                    exponentiated by the caller in float64 for bit-reproducible
                                    projections */
} ludvig_scene_opts;

/* Creates a scene from n Gaussians (Sec. 3.1: mean, covariance from scale and
 * rotation, opacity).  All inputs are device arrays and are COPIED:
 *   means [n,3], scales [n,3] (log or linear standard deviations, see opts),
 *   quats [n,4] (w,x,y,z; any non-zero norm), opacity [n] (in (0,1)).
 * n may be 0; opts may be NULL.  The per-Gaussian 3D covariance is
 * precomputed on `stream`.  *out receives the handle; destroy it with
 * ludvig_scene_destroy. */
ludvig_status ludvig_scene_create(const float* means, const float* scales, const float* quats,
                                  const float* opacity, int64_t n, const ludvig_scene_opts* opts,
                                  void* stream, ludvig_scene_t* out);

/* Waits for the scene's last asynchronous uplift call (if any), completes it
 * and returns its device status word (cleared afterwards): LUDVIG_OK, or
 * LUDVIG_ERR_TIMEOUT if a bounded wait of a kernel expired.  Groups of views
 * whose (tile, Gaussian) pairs or weight rows did not fit the scene's
 * workspace added nothing on the device; they are redone here, synchronously,
 * after the workspace has grown to fit them (later calls then fit).  Blocks
 * the calling thread. */
ludvig_status ludvig_sync(ludvig_scene_t scene);

/* Frees the scene and its workspace (synchronises the device). */
ludvig_status ludvig_scene_destroy(ludvig_scene_t scene);

/* Number of Gaussians of a scene. */
int64_t ludvig_scene_size(ludvig_scene_t scene);

/* Device bytes the scene's workspace holds now (it grows to the largest call
 * the scene has run); -1 for a NULL scene.  Safe to call from any thread,
 * also while a call on the scene runs (the figure may then be about to grow):
 * a server's admission can charge its resident scenes' workspaces against a
 * memory budget. */
int64_t ludvig_scene_workspace_bytes(ludvig_scene_t scene);

/* Uplifting, accumulation half (Sec. 3.2, Eq. 3; matrix form Eq. 5):
 *   num[i,:] += sum_{v,p} w_i(v,p) F_v[p,:]      den[i] += sum_{v,p} w_i(v,p)
 * over the n_views cameras `cams` (host [n_views]) of one image size
 * width x height (each <= 65535*16), with features `feats`
 * (device [n_views, height, width, d], channels-last, dtype `dtype`,
 * 1 <= d <= 65536; num 16-byte aligned when d % 4 == 0).
 * num (device [n,d] float32) and den (device [n] float32) are ADDED to, so
 * partial sums over disjoint view sets can be merged by addition (view
 * sharding, checkpoint/resume).  Summation order on the GPU is not fixed
 * (atomics), so results are reproducible only to rounding.
 * Where the products run: d <= 4 in the compositing pass itself (each weight
 * row, split into bfloat16 terms as below, is dotted with the tile's features
 * on CUDA cores as it is made); 4 < d < 32, or 32 <= d <= 512 with d % 8 == 0,
 * on the tensor cores (4 < d < 32 on features the library zero-pads to 32
 * channels in its workspace), float32 features as split-bfloat16 terms
 * (float32-level accuracy; LUDVIG_OPT_F32_TENSOR_CORES = 0 moves them, and
 * float32 d <= 4, to CUDA cores), bfloat16 features with the weights rounded
 * to bfloat16 for the product; any other d on CUDA cores with float32 weights.
 * Asynchronous: num/den are complete once ludvig_sync(scene) has returned
 * LUDVIG_OK (the views run in groups of up to 128; a group's projection, sorts
 * and weights overlap the previous group's products on two internal streams
 * that are joined back into `stream`). */
ludvig_status ludvig_uplift_accumulate(ludvig_scene_t scene, const ludvig_camera* cams,
                                       int32_t n_views, int32_t width, int32_t height,
                                       const void* feats, int32_t dtype, int32_t d,
                                       float* num, float* den, void* stream);

/* Uplifting, normalisation half (Eq. 3, D^-1 of Eq. 5):
 *   out[i,:] = num[i,:] / den[i] if den[i] > 0 else 0;  beta[i] = den[i].
 * num/out may alias (in place); beta may be NULL.  Device arrays. */
ludvig_status ludvig_uplift_finalize(int64_t n, int32_t d, const float* num, const float* den,
                                     float* out, float* beta, void* stream);

/* Full uplift f = D^-1 W^T F (Eq. 5): zeroes out (used as the numerator),
 * accumulates every view and normalises in place.  out: device [n,d] float32;
 * beta: device [n] float32 (beta_i = sum of weights, the importance score of
 * Sec. 3.2 "Gaussian filtering") or NULL.  Asynchronous like
 * ludvig_uplift_accumulate: out/beta are final once ludvig_sync(scene) has
 * returned LUDVIG_OK. */
ludvig_status ludvig_uplift(ludvig_scene_t scene, const ludvig_camera* cams, int32_t n_views,
                            int32_t width, int32_t height, const void* feats, int32_t dtype,
                            int32_t d, float* out, float* beta, void* stream);

/* The same uplift from HOST memory: feats is host [n_views,height,width,d]
 * (pinned memory gives full copy bandwidth), out host [n,d] and beta host [n]
 * or NULL.  Views are streamed to the device in chunks through a double
 * buffer that overlaps copies with compute; the call returns after the
 * results are back in host memory (it synchronises `stream`, and reports a
 * kernel-side status itself). */
ludvig_status ludvig_uplift_host(ludvig_scene_t scene, const ludvig_camera* cams, int32_t n_views,
                                 int32_t width, int32_t height, const void* feats, int32_t dtype,
                                 int32_t d, float* out, float* beta, void* stream);

/* FP8-E4M3 storage of features (the precision form's 8-bit variant; the
 * OCP 8-bit floating point format: bias 7, 3 mantissa bits, largest finite
 * value 448, no infinities).  Per view v of n_views views of view_elems
 * values each (feats device, float32 or bfloat16 by `dtype`):
 *   s_v = max |x| / 448 over the view (float32; 1 for an all-zero view),
 *   q   = E4M3 code of x / s_v (IEEE float32 division, round to nearest
 *         even, saturating at 448).
 * q: device uint8 [n_views * view_elems], 4-byte aligned; scales: device
 * float32 [n_views] (also the scratch of the per-view maximum).
 * n_views <= 65535. */
ludvig_status ludvig_fp8_quantize(const void* feats, int32_t dtype, int32_t n_views, int64_t view_elems,
                                  uint8_t* q, float* scales, void* stream);

/* Uplift (Eq. 5) of FP8-E4M3 features: the features are decode(q) * s_v
 * (q: device [n_views, height, width, d] codes, 4-byte aligned; scales:
 * device [n_views] float32, as ludvig_fp8_quantize writes them), each
 * rounded to bfloat16 (the E4M3 value times s_v) and uplifted by the
 * bfloat16 path, so results carry the bfloat16 bar on the decoded values.
 * With d % 16 == 0, 32 <= d <= 512 and q 16-byte aligned the aggregation
 * reads the codes themselves and decodes them in shared memory (one byte
 * per value crosses DRAM); otherwise each group of views (up to 128) is decoded
 * into the scene's workspace first.  out, beta as for ludvig_uplift. */
ludvig_status ludvig_uplift_fp8(ludvig_scene_t scene, const ludvig_camera* cams, int32_t n_views,
                                int32_t width, int32_t height, const uint8_t* q, const float* scales,
                                int32_t d, float* out, float* beta, void* stream);

/* One job of ludvig_uplift_batch: the arguments of one ludvig_uplift call
 * (same meaning, layout and rules). */
typedef struct {
    ludvig_scene_t scene;
    const ludvig_camera* cams;   /* host [n_views] */
    int32_t n_views, width, height;
    const void* feats;           /* device [n_views, height, width, d] */
    int32_t dtype, d;
    float* out;                  /* device [n, d] float32 */
    float* beta;                 /* device [n] float32 or NULL */
} ludvig_uplift_job;

#define LUDVIG_MAX_BATCH_SLOTS 32

/* Batched uplift: n_jobs independent uplifts of uneven size (each exactly
 * ludvig_uplift with the job's arguments, Eq. 5) sharing the GPU.
 * Jobs on the tensor-core path (packed_supported: bfloat16 features, float32
 * with LUDVIG_OPT_F32_TENSOR_CORES, any d < 32) with the same dtype, d and
 * image size whose feature buffers lie a whole number of views apart (as
 * slices of one feature array do) form a class: the class's views are
 * packed, largest scene first, into common groups of up to 128 views of
 * several jobs, so every stage launch serves many jobs.  The group size (the
 * per-view Gaussian scratch bound of a group) is picked per class: with
 * LUDVIG_OPT_BATCH_TUNE = 1 (default) by timing candidate sizes (256 MiB ..
 * 2 GiB) on up to 4 of the class's jobs (spread over its scene sizes) and 64
 * of their views each, into scratch outputs, the first time the process meets the class (dtype, d, image size,
 * log2 of the mean scene size), and kept for later batches; else
 * LUDVIG_OPT_GROUP_MB.  A packed group also holds at most bound / 32 pixels
 * (bound / 64 for float32: its weight rows grow with its pixels).  A class
 * that runs out of device memory is redone with half the bound (down to
 * 64 MiB).  The classes run one after another, largest first, on one
 * pooled context (its own workspace and two streams) driven by the calling
 * thread; the other jobs run as ludvig_uplift calls on `slots` host threads
 * (the calling thread joins them after the classes) with pooled workspaces
 * lent to their scenes.  1 <= slots <=
 * LUDVIG_MAX_BATCH_SLOTS.
 * Every job's work is ordered after the work already on `stream`, and
 * `stream` waits for all of it: to the caller the batch is one call on
 * `stream`.  A scene may appear in one job only (LUDVIG_ERR_ARG otherwise);
 * jobs may share feature buffers (read-only) but not outputs.  A job whose
 * arguments ludvig_uplift would reject fails alone.
 * job_status: host [n_jobs] or NULL, receives each job's status (a failure
 * inside a class fails the class's jobs).  Returns LUDVIG_OK when every job
 * succeeded, else the status of the first failing job in job order
 * (ludvig_last_error() names it); the other jobs still run.
 * Results equal those of the jobs run one by one, to float32 rounding
 * (summation order is not fixed).
 * Workspace: the contexts and slot workspaces come from a process-wide pool
 * (the scenes' own workspaces are left as they were), so device scratch
 * grows with `slots`, not with n_jobs; the pool keeps them for later
 * batches.  The call returns after every job's work has finished. */
ludvig_status ludvig_uplift_batch(const ludvig_uplift_job* jobs, int32_t n_jobs, int32_t slots,
                                  int32_t* job_status, void* stream);

/* One class of the last ludvig_uplift_batch call on any thread. */
typedef struct {
    int32_t dtype, d, width, height;
    int32_t jobs, views;
    int32_t groups;        /* groups formed: launches of each pipeline stage (-1: the single calls) */
    int32_t group_mb;      /* the groups' scratch bound, MiB */
    int32_t tuned;         /* 1: group_mb was picked by the tuner */
    int32_t redone;        /* groups that outgrew the workspace and were run again */
    int32_t workspace_mb;  /* device workspace of the class's context afterwards, MiB */
    float ms;              /* host time of the class (tuning included), ms */
} ludvig_batch_class;

/* Copies up to cap classes of the last batch into out (host, may be NULL) and
 * returns how many it had: the packed classes, then one entry (groups = -1)
 * for the jobs run as single calls. */
int32_t ludvig_batch_last_plan(ludvig_batch_class* out, int32_t cap);

/* Forgets the tuner's choices (the next batch times its classes again). */
ludvig_status ludvig_batch_forget_tuning(void);

/* Frees the idle pooled workspaces and contexts of ludvig_uplift_batch on the
 * current device (those of batches still running stay). */
ludvig_status ludvig_batch_release_workspaces(void);

/* Rendering of per-Gaussian features into views (Sec. 3.2, Eq. 4, F_hat = W f,
 * the operator whose transpose the uplift applies):
 *   out[v, y, x, :] = sum_i w_i(v, p) f[i, :]      p = pixel (x, y) of view v
 * with the weights of Eq. 1 (the same walk, rules and float32 decisions as the
 * uplift), no normalisation and no background term.
 *   f:   device [n, d] float32 (e.g. uplifted features), 16-byte aligned when
 *        d % 8 == 0 and 32 <= d <= 512 (the tensor-core path);
 *   out: device [n_views, height, width, d] float32, OVERWRITTEN: pixels
 *        without a contributor get 0.
 * d in [1, 65536].  With LUDVIG_OPT_F32_TENSOR_CORES = 1 (default) and
 * d % 8 == 0, 32 <= d <= 512, the products run on the tensor cores with
 * split-bfloat16 operands (float32-level accuracy); otherwise on CUDA cores in
 * float32.  Summation order is fixed (results are deterministic).
 * LUDVIG_ERR_TIMEOUT if a bounded wait of the tensor-core kernel expired. */
ludvig_status ludvig_render(ludvig_scene_t scene, const ludvig_camera* cams, int32_t n_views,
                            int32_t width, int32_t height, const float* f, int32_t d, float* out,
                            void* stream);

/* Gaussian filtering by importance (Sec. 3.2, "Gaussian filtering"; Sec. 4
 * keeps half of the Gaussians): beta_i, the sum of Gaussian i's rendering
 * weights over the training views (the beta output of the uplift), ranks the
 * Gaussians.  Writes the indices of the `keep` Gaussians with the largest
 * beta_i, ties to the lower index, in ascending order.
 *   beta: device [n] float32 (n = the scene's size); values <= 0 and NaN rank
 *         as 0;
 *   kept: device [keep] int32, written.
 * 0 <= keep <= n (keep = n - n/2 keeps the half the paper keeps).  The result
 * is exact given beta (an integer decision on the float32 values). */
ludvig_status ludvig_beta_select(ludvig_scene_t scene, const float* beta, int64_t keep, int32_t* kept,
                                 void* stream);

/* A new scene holding Gaussians idx[0..m) of `scene` (device int32 indices in
 * [0, n); repeats allowed), in that order: the filtered scene that later
 * uplifts and renders run on.  The precomputed covariances are copied, so each
 * Gaussian projects exactly as in the source scene.  Synchronises `stream`
 * (reads back an index check); LUDVIG_ERR_ARG if an index is out of range.
 * *out receives the handle (ludvig_scene_destroy frees it); the source scene
 * is unchanged. */
ludvig_status ludvig_scene_subset(ludvig_scene_t scene, const int32_t* idx, int64_t m, void* stream,
                                  ludvig_scene_t* out);

/* Relevancy of uplifted CLIP features to text queries (appendix, "Relevancy
 * scores", after LERF):
 *   r[i, q] = min_k exp(T s_iq) / (exp(T s_iq) + exp(T s_ik))
 * with s_iq = f^_i . phi^_q, s_ik = f^_i . phi^_{n_queries + k}, every vector
 * l2-normalised inside (a zero feature scores 1/2).
 *   feats: device [n, d] float32; phi: device [n_queries + n_canon, d]
 *   float32, the queries first, then the canonical phrases ("object",
 *   "things", "stuff", "texture" in the paper); r: device [n, n_queries].
 * 1 <= n_queries, 1 <= n_canon, n_queries + n_canon <= 64 and
 * (n_queries + n_canon) * d <= 49152; temperature > 0 (the paper's T = 10). */
ludvig_status ludvig_relevancy(const float* feats, int64_t n, int32_t d, const float* phi, int32_t n_queries,
                               int32_t n_canon, float temperature, float* r, void* stream);

/* ---- tracing ------------------------------------------------------------ */

/* Stages of the path, as reported by ludvig_trace_read. */
typedef enum {
    LUDVIG_STAGE_PROJECT = 0,     /* EWA projection, depth keys, tile rectangles */
    LUDVIG_STAGE_DEPTH_SORT = 1,  /* radix sort of depths per view */
    LUDVIG_STAGE_BIN = 2,         /* tiles-touched scan and pair emission */
    LUDVIG_STAGE_TILE_SORT = 3,   /* radix sort of (view, tile) pairs and tile ranges */
    LUDVIG_STAGE_COMPOSITE = 4,   /* compositing weights + aggregation (the hot kernel) */
    LUDVIG_STAGE_NORMALISE = 5,
    LUDVIG_STAGE_KNN = 6,
    LUDVIG_STAGE_GRAPH = 7,       /* union edges, weights, normalisation */
    LUDVIG_STAGE_DIFFUSE = 8,
    LUDVIG_STAGE_WEIGHTS = 9,     /* inside COMPOSITE: tensor-core path, compositing weights */
    LUDVIG_STAGE_AGGREGATE = 10,  /* inside COMPOSITE: tensor-core path, W F products into num/den */
    LUDVIG_STAGE_RENDER = 11,     /* ludvig_render, stage 6: weights + W f products */
    LUDVIG_STAGE_RENDER_PRODUCT = 12, /* inside RENDER: the W f products alone */
    LUDVIG_STAGE_FILTER = 13,     /* ludvig_beta_select, ludvig_topfrac_positive */
    LUDVIG_STAGE_RELEVANCY = 14,  /* ludvig_relevancy */
    LUDVIG_STAGE_COUNT = 15
} ludvig_stage;

typedef struct {
    double ms[16];              /* summed device time per stage (CUDA events) */
    int64_t calls[16];          /* timed intervals per stage */
    int64_t kernel_launches;    /* kernels launched by the library */
} ludvig_trace;

/* Turns stage tracing on or off for the whole process (off by default).
 * While on, every stage is bracketed by CUDA events recorded on the stream
 * the stage runs on; the launch counter always runs. */
ludvig_status ludvig_trace_enable(int32_t on);

/* Waits for the recorded events, adds their durations into *out and, if
 * reset != 0, clears the trace and the launch counter. */
ludvig_status ludvig_trace_read(ludvig_trace* out, int32_t reset);

/* ---- inspection entry points (used by the parity tests) ---------------- */

/* Per-Gaussian float32 projection of one view (device outputs):
 *   rec [n,8]: mean2d.x, mean2d.y, depth, conic a, b, c, opacity, radius
 *   rect [n,4]: tile rectangle x0,y0,x1,y1 (half-open; all 0 when culled). */
ludvig_status ludvig_debug_project(ludvig_scene_t scene, const ludvig_camera* cam, int32_t width,
                                   int32_t height, float* rec, int32_t* rect, void* stream);

/* Depth-ordered per-tile lists of one view.  pruned = 0: every Gaussian whose
 * tile rectangle covers the tile (the 3DGS binning rule); pruned = 1: the
 * lists the uplift walks, which additionally drop Gaussians whose
 * alpha >= 1/255 ellipse cannot reach any pixel centre of the tile (such a
 * Gaussian is skipped at every pixel of the tile, so no weight changes).
 * ranges: device [ntiles,2] int64 [start,end) into list; list: device int32
 * [cap].  *total (host) receives the list length; the list is written only
 * when total <= cap.  Synchronises `stream`. */
ludvig_status ludvig_debug_tile_lists(ludvig_scene_t scene, const ludvig_camera* cam,
                                      int32_t width, int32_t height, int32_t pruned,
                                      int64_t* ranges, int32_t* list, int64_t cap, int64_t* total,
                                      void* stream);

/* Per-pixel float32 transmittance after the compositing walk of one view
 * (device [height,width]) and the number of contributors (device int32). */
ludvig_status ludvig_debug_transmittance(ludvig_scene_t scene, const ludvig_camera* cam,
                                         int32_t width, int32_t height, float* t_final,
                                         int32_t* n_contrib, void* stream);

/* Tensor-core product used by the bfloat16 aggregation, on one 16x16 tile:
 *   out[r, c] = sum_{p < 256} a[r, p] * f[p, c]      (r < 128, c < d)
 * a: device [128,256] bfloat16 row-major (a W tile: Gaussian x pixel),
 * f: device [16,16,d] bfloat16 (a feature tile, pixel p = 16*y + x),
 * out: device [128,d] float32; d in {64, 128, ..., 512}.  Synchronises. */
ludvig_status ludvig_debug_mma_bf16(const void* a, const void* f, int32_t d, float* out, void* stream);

/* Failure-detection check of the bounded waits (the paper has no
 * counterpart): one kernel waits on an mbarrier that nothing arrives on, with
 * the same expiry logic the tensor-core kernels use but a budget of `cycles`
 * SM clock cycles (0 .. 4e9; the kernels' own budget is 4e9, about 2 s).
 * When it expires the kernel records LUDVIG_ERR_TIMEOUT in a status word and
 * returns; nothing traps or faults, so the context stays usable.  Returns
 * that status (LUDVIG_ERR_TIMEOUT) with *waited (may be NULL) = the cycles
 * waited.  Synchronises `stream`. */
ludvig_status ludvig_debug_wait_timeout(int64_t cycles, int64_t* waited, void* stream);

/* Failure-detection check of the asynchronous status path (the paper has no
 * counterpart): enqueues on `stream` one kernel that waits on an mbarrier that
 * nothing arrives on, with the expiry logic of the tensor-core kernels and a
 * budget of `cycles` SM clock cycles (0 .. 4e9).  On expiry it records
 * LUDVIG_ERR_TIMEOUT in the scene's device status word, as a kernel of an
 * asynchronous uplift would, and returns; nothing traps.  The call itself
 * returns without waiting; ludvig_sync(scene) then reports the status. */
ludvig_status ludvig_debug_scene_timeout(ludvig_scene_t scene, int64_t cycles, void* stream);

/* ---- graph diffusion (Sec. 3.3) ----------------------------------------- */

/* Exact k nearest neighbours of every Gaussian centre (Euclidean; the point
 * itself excluded; squared distances on float32 as (dx*dx+dy*dy)+dz*dz with
 * d = x_j - x_i; equal distances to the lower index; missing neighbours -1).
 * nbr: device [n,k] int32.  1 <= k <= 64. */
ludvig_status ludvig_knn(ludvig_scene_t scene, int32_t k, int32_t* nbr, void* stream);

/* Builds the diffusion graph: the union edge set {i,j : j in N_k(i) or
 * i in N_k(j)} (Sec. 3.3) with weight
 *   A_ij = exp(-||mu_i - mu_j||^2 / spatial_h) * max(0, cos(f_i, f_j))
 * (f: device [n,df] float32 per-Gaussian features, e.g. uplifted DINOv2;
 * a zero vector has cosine 0), optionally row-normalised (A <- D_A^-1 A, rows
 * summing to 0 stay 0).  If binarize > 0 weights above it become 1 and the
 * others 0 before normalisation.  The graph (CSR, float32) lives on the
 * device until ludvig_graph_destroy. */
ludvig_status ludvig_graph_build(ludvig_scene_t scene, int32_t k, const float* feats, int32_t df,
                                 float spatial_h, float binarize, int32_t row_normalize,
                                 void* stream, ludvig_graph_t* out);

ludvig_status ludvig_graph_destroy(ludvig_graph_t graph);

/* Number of stored (directed) edges of the graph. Synchronises nothing. */
int64_t ludvig_graph_nnz(ludvig_graph_t graph);

/* Device bytes the graph's workspace holds now (diffusion scratch, the sliced
 * matrix copy); -1 for a NULL graph.  Same rules as
 * ludvig_scene_workspace_bytes. */
int64_t ludvig_graph_workspace_bytes(ludvig_graph_t graph);

/* Copies the CSR arrays to device buffers: row_ptr [n+1] int64, col [nnz]
 * int32, val [nnz] float32 (columns sorted within each row). */
ludvig_status ludvig_graph_export(ludvig_graph_t graph, int64_t* row_ptr, int32_t* col, float* val,
                                  void* stream);

/* Graph diffusion (Sec. 3.3, Eq. 8) on every column of x0 (device [n,dx]):
 *   g_0 = x0,  g_{t+1} = A (g_t / ||g_t||_2),  t < iters.
 * out: device [n,dx]; must not alias x0.  A column whose norm is 0 stays 0.
 * 1 <= dx <= 32.  With dx = 1 the steps run on a sliced copy of the matrix
 * (32-row slices, column-major) that the first call after the graph's values
 * change builds in the graph's workspace; that call synchronises `stream`
 * once. */
ludvig_status ludvig_diffuse(ludvig_graph_t graph, const float* x0, int32_t dx, int32_t iters,
                             float* out, void* stream);

/* ---- paper-form diffusion (Eq. 7 with the appendix's S_f and P; Sec. 4.1) --
 *
 * The RBF similarity S_f(f_i, f_j) = exp(-||f^_i - f^_j||^2 / (b s_f^2)) of
 * l2-normalised features, with s_f the median of the pairwise distances,
 * read as the median over the graph's edges (all n^2 pairs are out of reach;
 * the mean of the two middle values for an even edge count); the unary term
 * P(f_i) = S_f(f_i, f_bar) (scribble form: f_bar the normalised mean of the
 * anchors' normalised features, its own bandwidth); A_ij = S_f P_i^1/2
 * P_j^1/2, thresholded at 1e-5 for segmentation; g_0 the top 10 % of the
 * uplifted reference mask's positive values; h_i = P_i on the nodes g_T
 * reaches after T steps, 0 elsewhere.  The scene part (kNN, edge distances,
 * s_f) is built once; the prompt part (P, A, h) per query. */

/* The union kNN graph of ludvig_graph_build (same edges) for the RBF
 * similarity: keeps ||f^_i - f^_j||^2 per edge (float32, from the cosine of
 * the two rows: 2 - 2 cos, 1 with one zero row, 0 with two) and s_f, the
 * median edge distance; values are S_f with b = 1 and no unary term until
 * ludvig_graph_reweight (0 when s_f = 0, e.g. identical features: the RBF
 * similarity is then undefined).  feats: device [n, df] float32.
 * Synchronises. */
ludvig_status ludvig_graph_build_rbf(ludvig_scene_t scene, int32_t k, const float* feats, int32_t df,
                                     void* stream, ludvig_graph_t* out);

/* s_f of an RBF graph (host float). */
ludvig_status ludvig_graph_feature_scale(ludvig_graph_t graph, float* s_f);

/* Values of an RBF graph for a prompt: A_ij = exp(-d2_ij / (b s_f^2))
 * sqrt(P_i P_j) (unary: device [n] or NULL for P = 1), then, if binarize > 0,
 * 1 where A_ij > binarize and 0 elsewhere, then, if row_normalize, each row
 * divided by its sum (zero rows stay zero).  LUDVIG_ERR_ARG when s_f = 0. */
ludvig_status ludvig_graph_reweight(ludvig_graph_t graph, float bandwidth, const float* unary, float binarize,
                                    int32_t row_normalize, void* stream);

/* Unary term of the scribble form: P_i = exp(-||f^_i - f_bar||^2 / (b s_f^2))
 * with the graph's s_f and f_bar the l2-normalised sum of f^_i over the anchor
 * nodes {i : g0_i > 0} (zero without anchors).  feats: device [n, df]
 * float32 (the graph's features); g0: device [n]; unary: device [n], written. */
ludvig_status ludvig_unary_anchor(ludvig_graph_t graph, const float* feats, int32_t df, const float* g0,
                                  float bandwidth, float* unary, void* stream);

/* g_0 of the segmentation task: g0_i = u_i on the ceil(npos * percent / 100)
 * Gaussians with the largest positive u_i (ties to the lower index; npos =
 * the number of u_i > 0), 0 elsewhere.  u, g0: device [n] float32 (n = the
 * scene's size); 0 <= percent <= 100. */
ludvig_status ludvig_topfrac_positive(ludvig_scene_t scene, const float* u, int32_t percent, float* g0,
                                      void* stream);

/* Segmentation weight after `steps` diffusion steps: S = {i : g_T,i > 0}, which
 * for A >= 0 and g_0 >= 0 is the set reached from {i : g0_i > 0} by walks of
 * exactly `steps` edges with A_ij > 0 (computed as that walk on bit sets, so
 * no float underflow can lose a node), then h_i = P_i on S (1 when unary is
 * NULL) and 0 elsewhere.  g0, h: device [n, dx] (column q = query q), 1 <= dx
 * <= 32; unary: device [n] or NULL.  Negative g0 entries count as not
 * reached. */
ludvig_status ludvig_reach_weight(ludvig_graph_t graph, const float* g0, int32_t dx, int32_t steps,
                                  const float* unary, float* h, void* stream);

/* Graph diffusion that allocates no memory (the paper has no counterpart: this
 * is a service entry point).  It computes what ludvig_diffuse
 * computes, for callers that must not allocate device memory: a request loop
 * that runs under a strict no-allocation policy once it is warm, or a process
 * whose device memory is already handed out to another allocator.  Its
 * scratch (the ping-pong vector
 * and the per-step norms) lives in statically allocated device memory of the
 * library: at most 1,048,576 elements (n * dx) and at most 1024 steps; larger
 * requests fail with LUDVIG_ERR_ARG before anything is enqueued.  Every GPU
 * that loads the library holds this scratch (about 4.3 MB) until the process
 * exits.  The first call on a device translates the scratch's address for
 * that device (once per device, with the device current); make that first
 * call before any stream capture.  All calls share the one scratch area, so
 * calls whose work overlaps on the GPU (different streams, or different host
 * threads without ordering) race; the call clears the norm slots it uses.
 * Arguments, layouts and results are those of ludvig_diffuse (to float32
 * rounding: it keeps the CSR kernel, whose summation order within a row
 * differs from the sliced one). */
ludvig_status ludvig_diffuse_noalloc(ludvig_graph_t graph, const float* x0, int32_t dx, int32_t iters,
                                     float* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LUDVIG_H */
