/*
 * ba.h - C ABI of the B300 bundle-adjustment library (libba.so).
 *
 * The library runs the Levenberg-Marquardt bundle-adjustment iteration of
 * cuSfM (arXiv 2510.15271, Sec. 4.3 "Iterative Triangulation and Mapping")
 * on one NVIDIA B300 GPU:
 *   minimise  F = 1/2 sum_k rho(|| pi(K T_cam(k) X_pt(k)) - p_obs,k ||^2)
 * over camera poses T (6-DoF, world -> camera) and points X, with the
 * reprojection error of Sec. 4.3 (reprojection equation), the robust loss
 * rho of the stage-one objective (Sec. 4.3, objective L; Huber here) and
 * the fixed-pose subsets of Sec. 4.3 (absolute pose constraints) applied as
 * a hard mask.  Each iteration: residuals + analytic Jacobians + IRLS Huber
 * weights, block accumulation, Schur complement of the point blocks, a
 * direct (dense Cholesky) or block-Jacobi PCG solve of the reduced camera
 * system, point back-substitution, trial step, gain ratio and damping
 * update, all on the device with no host synchronisation per iteration.
 *
 * Conventions (all calls):
 *   - Pose: 7 doubles (qw, qx, qy, qz, tx, ty, tz), a unit quaternion and a
 *     translation of the world -> camera map x_c = R X + t.  Camera axes: x
 *     right, y down, z forward.  Pixel: (fx x/z + cx, fy y/z + cy).
 *   - Every array is dense, row-major, native-endian, with no padding.
 *   - Inputs are copied in; the caller keeps ownership of every buffer it
 *     passes and may reuse it as soon as the call returns.  Outputs are
 *     written into caller buffers.
 *   - Every call returns a ba_status; on failure ba_last_error() describes
 *     the cause.  A handle is used by one host thread at a time.
 *   - mem_kind BA_MEM_HOST: pointers are host memory (pinned or pageable).
 *     BA_MEM_DEVICE: pointers are device memory of the handle's device,
 *     read (or written) in stream order on the handle's stream.
 */
#ifndef BA_H
#define BA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ba_handle ba_handle;

typedef enum {
  BA_OK = 0,
  BA_ERR_INVALID_ARG = 1, /* bad pointer, size, index, non-finite value   */
  BA_ERR_OOM = 2,         /* device allocation failed                     */
  BA_ERR_CUDA = 3,        /* a CUDA runtime call failed                   */
  BA_ERR_NOT_READY = 4,   /* ba_poll: request still running               */
  BA_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up           */
  BA_ERR_BUSY = 6,        /* ba_submit: request table full                */
  BA_ERR_STATE = 7,       /* call out of order (e.g. solve before set)    */
  BA_ERR_NUMERIC = 8      /* non-finite cost or state after the solve     */
} ba_status;

enum { BA_FP64 = 0, BA_FP32 = 1 };                          /* precision  */
enum { BA_SOLVER_AUTO = 0, BA_SOLVER_DENSE = 1, BA_SOLVER_PCG = 2 };
enum { BA_MEM_HOST = 0, BA_MEM_DEVICE = 1 };

/* Optional device allocator (for example PyTorch's caching allocator).  When
 * alloc is NULL the library uses cudaMalloc / cudaFree.  alloc returns NULL
 * on failure; stream is the handle's cudaStream_t. */
typedef void* (*ba_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*ba_free_fn)(void* ptr, void* ctx);

typedef struct {
  int precision;        /* BA_FP64: every step in FP64.  BA_FP32: residuals,
                           Jacobians, Schur blocks and PCG in FP32; cost sum,
                           gain ratio, damping and 3x3 point inverses FP64.   */
  int solver;           /* BA_SOLVER_DENSE: Cholesky of the reduced camera
                           system; BA_SOLVER_PCG: block-Jacobi PCG;
                           BA_SOLVER_AUTO: dense when 6C <= dense_max_dim.    */
  int max_lm_iters;     /* LM iterations (one solve + one trial each), 1..256 */
  double huber_delta;   /* Huber threshold in px; <= 0: plain least squares   */
  double pcg_tol;       /* stop when ||r|| <= pcg_tol ||b||                    */
  int pcg_max_iters;    /* cap on products with S per solve (per inner solve) */
  int refine;           /* PCG: iterative refinement on the FP64 residual
                           b - S x (with BA_FP64 this is PCG restarted from
                           the current iterate)                               */
  int refine_max;       /* outer refinement steps (default 5)                 */
  double refine_tol;    /* stop refinement at ||b - S x|| <= tol ||b||        */
  double mu0;           /* initial damping (default 1e-4)                     */
  int dense_max_dim;    /* BA_SOLVER_AUTO threshold on 6C (default 1200)      */
  int device;           /* CUDA device ordinal                                */
  void* cuda_stream;    /* cudaStream_t to run on; NULL: library-owned stream */
  int use_graph;        /* replay the LM loop as one CUDA graph (default 1)   */
  ba_alloc_fn alloc;    /* optional device allocator                          */
  ba_free_fn free_fn;
  void* alloc_ctx;
  /* serving handles only (see ba_create_server) */
  size_t serve_arena_bytes; /* device memory reserved for request slots      */
  int serve_slots;          /* maximum requests resident at once             */
  int serve_queue;          /* maximum requests waiting for admission        */
  int profile;              /* record per-kernel device times (CUDA events
                               between the kernels of the captured loop)      */
  int pcg_variant;          /* PCG kernel.  0: auto (2 when the reduced
                               system stays in shared memory and there is no
                               refinement, 4 when it does not stay resident,
                               else 1); 1: standard PCG on a cooperative grid
                               (two grid barriers per iteration); 2:
                               pipelined PCG (one grid barrier per iteration,
                               recurrence vectors in FP64); 3: standard
                               PCG in one thread-block cluster (hardware
                               cluster barriers, exchanges through
                               distributed shared memory; falls back to 1
                               when S does not fit, or with refinement); 4:
                               standard PCG with S streamed through shared
                               memory by bulk copies, one CTA per SM and the
                               same number of blocks of S per CTA (falls back
                               to 1 when its plan does not fit); 5: the same
                               with one fused reduction per iteration (the
                               same iterates in exact arithmetic; measured
                               slower on this part: seven FP64 dot products
                               per iteration cost more than the grid barrier
                               they save)                                    */
  double mu_min;            /* floor of the damping used in the linear system;
                               < 0: auto (1e-4 for BA_FP32, where rounding in
                               the FP32 Schur complement otherwise exceeds its
                               smallest eigenvalues; 0 for BA_FP64)          */
  double serve_tick_ms;     /* serving handles: every resident request gets one
                               LM iteration per tick, and more while the tick
                               is younger than this (ms; 0: exactly one; < 0:
                               auto, 90 % of the previous tick, >= 2 ms)      */
  double serve_split_ms;    /* serving handles: a request whose whole solve is
                               estimated to take longer than this (ms, on one
                               SM) runs to completion in a launch of its own
                               beside the ticks instead of in them; < 0: every
                               request in the ticks; 0: none.  Up to 16 such
                               launches run at once, each on its own stream:
                               give the process CUDA_DEVICE_MAX_CONNECTIONS
                               >= 20 (read when the CUDA context is created)
                               so that they do not share hardware queues with
                               the ticks, which would hold a tick behind a
                               long launch                                   */
  double prior_seq_weight;  /* lambda_c of the sequential pose prior (Sec. 4.2,
                               Eq. seq, adjacent frames; 0: off): adds
                               1/2 lambda_c sum_i ||T_cw,i+1 T_wc,i - Q_i||^2,
                               Q_i the relative pose of cameras i, i+1 (in
                               index order) in the state given to
                               ba_set_problem; Frobenius norm of the top 3x4
                               blocks.  ba_solve only                         */
  double prior_abs_weight;  /* lambda_a of the absolute pose prior (Sec. 4.3,
                               Eq. abs; 0: off): adds 1/2 lambda_a sum_i
                               ||T_wc,i - T_wc,i^0||^2 with T_wc^0 the
                               camera-to-world pose given to ba_set_problem.
                               ba_solve only (ba_solve_batch and
                               ba_create_server refuse it)                    */
  int pcg_resident_cap;     /* bytes of shared memory per CTA in which the PCG
                               kernels may keep their rows of S resident
                               (0: the device's limit).  A small cap makes
                               them read S from global memory every product,
                               as on systems too large to stay resident; for
                               tests and tuning                               */
} ba_options;

typedef struct {
  double fx, fy, cx, cy;  /* pinhole intrinsics in px, shared by all cameras */
} ba_intrinsics;

#define BA_MAX_ITERS 256

/* Per-solve report.  cost[0] is F at the initial state, cost[i+1] F after
 * iteration i (unchanged by a rejected step). */
typedef struct {
  int32_t status;                    /* ba_status of the solve               */
  int32_t n_iters;
  int32_t n_accepted;
  int32_t solver;                    /* BA_SOLVER_DENSE or BA_SOLVER_PCG     */
  double cost[BA_MAX_ITERS + 1];
  uint8_t accepted[BA_MAX_ITERS];
  double mu[BA_MAX_ITERS];           /* damping used by iteration i's solve  */
  int32_t pcg_iters[BA_MAX_ITERS];   /* products with S (0 for dense)       */
  double pcg_rel_residual[BA_MAX_ITERS];
  double gain[BA_MAX_ITERS];         /* gain ratio; -inf when dL <= 0        */
  double rmse_px;                    /* final sqrt(sum ||r||^2 / n_valid)    */
  int64_t n_valid_obs;               /* observations with depth >= 1e-3     */
  double solve_ms;                   /* device time of the LM loop           */
  double setup_ms;                   /* device time of ba_set_problem        */
  int32_t n_kernels;                 /* library kernels launched by the solve */
  int32_t pcg_variant;               /* PCG kernel the solve ran (the values of
                                        ba_options.pcg_variant; 0: dense)     */
} ba_report;

/* Per-kernel device time of the last ba_solve (opts.profile = 1 only). */
typedef struct {
  char name[24];
  int32_t launches;
  int32_t pad;
  double total_ms;
} ba_kernel_stat;

/* Fill *opts with the defaults: FP64, AUTO solver, 10 iterations, no Huber,
 * PCG tol 1e-6 / 100, no refinement (5 steps, tol 1e-6 when enabled),
 * mu0 1e-4, dense_max_dim 1200, device 0, library stream, graphs on,
 * cudaMalloc, serving arena 0 (= 1/4 of free memory), 256 slots, 4096 queue,
 * tick 4 ms, split 10 ms, no pose priors. */
void ba_options_default(ba_options* opts);

/* Create a solver handle on opts->device.  *out receives the handle; the
 * handle owns every device buffer it allocates.  Errors: INVALID_ARG (NULL
 * pointers, bad option values), CUDA. */
ba_status ba_create(const ba_options* opts, ba_handle** out);

/* Load a problem (Sec. 4.3: poses, points, tracks of observations, fixed
 * camera subset) and build its device layout: observations sorted by
 * (camera, point) and by (point, camera), CSR indexes of both orders and the
 * block pattern of the reduced camera matrix S.  Replaces any earlier
 * problem on the handle.
 *   cam_qt   [n_cams][7]   initial poses (see conventions)
 *   pts      [n_pts][3]    initial points
 *   obs_cam  [n_obs]       camera index of each observation, 0..n_cams-1
 *   obs_pt   [n_obs]       point index of each observation, 0..n_pts-1
 *   obs_uv   [n_obs][2]    measured pixel (u, v)
 *   K                      intrinsics (host pointer always)
 *   cam_fixed [n_cams] or NULL: nonzero = pose held fixed (gauge / prior map)
 * Errors: INVALID_ARG when a size is < 1, an index is out of range, a value
 * is not finite, a quaternion is zero, a point has fewer than 2
 * observations or a free camera has none; OOM; CUDA. */
ba_status ba_set_problem(ba_handle* h, int32_t n_cams, int32_t n_pts, int64_t n_obs,
                         const double* cam_qt, const double* pts, const int32_t* obs_cam,
                         const int32_t* obs_pt, const double* obs_uv, const ba_intrinsics* K,
                         const uint8_t* cam_fixed, int mem_kind);

/* Run max_lm_iters LM iterations from the current state and wait for them.
 * The state left on the device is the last accepted one, so a second call
 * continues where the first stopped (resume).  out may be NULL.
 * Errors: STATE (no problem loaded), TIMEOUT (a device barrier gave up),
 * NUMERIC (non-finite cost), CUDA. */
ba_status ba_solve(ba_handle* h, ba_report* out);

/* Copy the current state out: cam_qt_out [n_cams][7] (qw >= 0), pts_out
 * [n_pts][3]; either may be NULL.  Errors: STATE, INVALID_ARG, CUDA. */
ba_status ba_get_state(const ba_handle* h, double* cam_qt_out, double* pts_out, int mem_kind);

/* Overwrite the state (poses, points) of the loaded problem, keeping its
 * layout; the damping restarts from mu0.  Errors: STATE, INVALID_ARG, CUDA. */
ba_status ba_set_state(ba_handle* h, const double* cam_qt, const double* pts, int mem_kind);

/* Diagnostic: the reduced camera system of the last linear solve of the
 * last ba_solve, as the device holds it, for checking the solve on the host
 * (host memory, FP64).  Rows and columns of fixed cameras are identity rows
 * with a zero right-hand side.
 *   dim    6 n_cams
 *   S_out  [dim][dim] or NULL: S = U* - W V*^-1 W^T as stored (in the path's
 *          precision, promoted), zero outside its block pattern
 *   b_out  [dim] or NULL: its right-hand side before rounding to the path's
 *          precision (-g_c + W V*^-1 g_p in FP64)
 *   x_out  [dim] or NULL: the solution the step used: the FP64 iterate of the
 *          refinement loop when refinement is on, else the solver's output
 *          in the path's precision, promoted
 * Errors: STATE (no finished solve), INVALID_ARG (dim), CUDA. */
ba_status ba_get_reduced_system(const ba_handle* h, int32_t dim, double* S_out, double* b_out,
                                double* x_out);

/* Kernel timings of the last solve, one entry per kernel kind: out[max]
 * receives up to max entries, *n the number written.  A serving handle adds
 * serve_tick (ticks, their summed milliseconds), serve_completed (requests),
 * serve_large (launches of long requests, their summed milliseconds) and
 * serve_tick_ctas (mean CTAs of a tick in launches, mean resident requests
 * of a tick in total_ms).  Errors: STATE (no solve yet or profiling off),
 * INVALID_ARG. */
ba_status ba_kernel_stats(const ba_handle* h, ba_kernel_stat* out, int32_t max, int32_t* n);

/* Reprojection cost F = 1/2 sum_k rho(||r_k||^2) of a given state, with no
 * device allocation.  The paper has no counterpart: this entry point exists
 * for callers that may not allocate device memory at the point of use (for
 * example a vehicle or robot process whose device memory plan is fixed at
 * start-up, or a host library that owns every allocation of its context
 * through its own pool).  It calls no cudaMalloc, cudaFree or allocating
 * library routine; its scratch is one file-scope device array of about
 * 1.5 MB.  The library's device code is loaded lazily, so the first call on
 * a device is where the driver loads the array and takes its memory; the
 * array is then held until the process exits.  Make that first call at
 * start-up (a one-camera problem will do), before any stream capture on the
 * device begins: it also looks up the array's device address, with that
 * device current, and later calls take no device memory at all.  The address
 * is kept per device and does not survive cudaDeviceReset: do not call this
 * entry point on a device after resetting it.
 *   device       CUDA device ordinal; the caller's current device is restored
 *   cuda_stream  cudaStream_t to run on (NULL: the legacy default stream)
 *   cam_qt, pts, obs_cam, obs_pt, obs_uv   device pointers, layouts as in
 *                ba_set_problem; observations in any order
 *   K            host pointer; huber_delta as in ba_options (<= 0: none)
 *   cost_out     device pointer to one double that receives F (unspecified
 *                when the call fails)
 * Observations with depth below 1e-3 leave the sum, as in ba_solve.  The call
 * blocks until cost_out is written.  Limits: n_cams <= 16384.  Every call on
 * a device shares the scratch array and keeps the last call's contents (the
 * call clears what must start at zero); calls whose work overlaps on the GPU
 * race.  Errors (message in ba_last_error(NULL)): INVALID_ARG (NULL pointer,
 * size < 1, n_cams above the limit, and, naming the first offender, an index
 * out of range, a non-finite pose, point or pixel, or a zero quaternion, as
 * ba_set_problem refuses them), CUDA (including a kernel that fails to
 * launch). */
ba_status ba_cost_noalloc(int device, void* cuda_stream, int32_t n_cams, int32_t n_pts,
                          int64_t n_obs, const double* cam_qt, const double* pts,
                          const int32_t* obs_cam, const int32_t* obs_pt, const double* obs_uv,
                          const ba_intrinsics* K, double huber_delta, double* cost_out);

/* Reprojection error of every observation and its outlier classification:
 * the step after each BA round of the paper's mapping loop (Sec. 4.3:
 * reprojection errors are computed from the updated points and poses, and
 * projections beyond the outlier threshold are removed).
 *   device, cuda_stream  CUDA device ordinal; stream to run on (NULL: the
 *                legacy default stream); the caller's current device is
 *                restored
 *   cam_qt [n_cams][7], pts [n_pts][3], obs_cam, obs_pt [n_obs],
 *   obs_uv [n_obs][2], K   as in ba_set_problem
 *   threshold_px the outlier threshold (>= 0)
 *   err2_out     [n_obs] or NULL: ||pi(K (R X + t)) - p_obs||^2 in px^2,
 *                +inf where the point's depth is below 1e-3
 *   inlier_out   [n_obs] or NULL: 1 where err2 <= threshold_px^2, else 0
 *   n_inliers    host pointer or NULL: the number of inliers
 *   mem_kind     BA_MEM_HOST: every array pointer is host memory (copied
 *                in and out through device scratch);
 *                BA_MEM_DEVICE: device memory of `device`
 * FP64 throughout.  Blocks until the outputs are written.  This call and
 * ba_triangulate keep their device scratch between calls (per device, grown
 * as needed, released at process exit) and serialise concurrent calls on one
 * device.  Errors (message
 * in ba_last_error(NULL)): INVALID_ARG (NULL input, sizes, threshold,
 * intrinsics, an index out of range), OOM, CUDA. */
ba_status ba_reprojection_errors(int32_t device, void* cuda_stream, int32_t n_cams, int32_t n_pts,
                                 int64_t n_obs, const double* cam_qt, const double* pts,
                                 const int32_t* obs_cam, const int32_t* obs_pt,
                                 const double* obs_uv, const ba_intrinsics* K,
                                 double threshold_px, double* err2_out, uint8_t* inlier_out,
                                 int64_t* n_inliers, int32_t mem_kind);

/* Triangulation of every point by the DLT of the paper's Sec. 4.3, Eq. (dlt),
 * from its observations whose mask is set, with the given camera poses: the
 * homogeneous point minimising the sum of ||P_j X - lambda_j p_j||^2, P_j =
 * [R_j | t_j] and p_j the observation in normalised camera coordinates
 * K^-1 (u, v, 1); that is the eigenvector of the smallest eigenvalue of A^T A,
 * A the two rows x P_j^3 - P_j^1, y P_j^3 - P_j^2 of each observation.
 *   obs_mask     [n_obs] or NULL (all observations): nonzero = use
 *   pts_out      [n_pts][3]: the triangulated points, NaN where status != 0
 *   status_out   [n_pts] or NULL: 0 triangulated; 1 fewer than 2 observations
 *                used; 2 the solution lies at infinity (|X_4| <= 1e-12 ||X||);
 *                3 behind a camera that observes it (depth below 1e-3)
 * Other arguments as in ba_reprojection_errors.  FP64; each point's rows are
 * summed in (point, camera) order, so results do not depend on the order of
 * the observations.  Blocks until the outputs are written.  Errors:
 * INVALID_ARG, OOM, CUDA. */
ba_status ba_triangulate(int32_t device, void* cuda_stream, int32_t n_cams, int32_t n_pts,
                         int64_t n_obs, const double* cam_qt, const int32_t* obs_cam,
                         const int32_t* obs_pt, const double* obs_uv, const ba_intrinsics* K,
                         const uint8_t* obs_mask, double* pts_out, int8_t* status_out,
                         int32_t mem_kind);

/* Self-test of the bounded grid barrier the PCG kernels wait at: launches
 * `blocks` co-resident CTAs (1..64) that meet at one grid barrier expecting
 * `expected` arrivals, each wait giving up after limit_ms (0 < limit_ms <=
 * 1000).  With expected > blocks the wait runs out: every CTA records the
 * time-out in the error word and returns, as the PCG kernels do, and the
 * device stays usable.  *timed_out receives 1 if the barrier timed out, 0 if
 * it completed; *waited_ms (may be NULL) the kernel's duration.  Blocks
 * until done; uses the legacy default stream of `device`, and restores the
 * caller's current device.  Errors (message in ba_last_error(NULL)):
 * INVALID_ARG, CUDA. */
ba_status ba_selftest_barrier(int32_t device, int32_t blocks, int32_t expected, double limit_ms,
                              int32_t* timed_out, double* waited_ms);

/* Release the handle and everything it owns.  NULL is ignored. */
void ba_destroy(ba_handle* h);

/* Description of the handle's last error ("" if none).  h may be NULL, then
 * the last error of a failed ba_create on this thread is returned. */
const char* ba_last_error(const ba_handle* h);

/* ------------------------------------------------------------------------ */
/* Batched and served local BA.                                             */

/* One independent problem (a local-BA window or a served request).  Arrays
 * are host memory; the *_out arrays (optional) receive the final state. */
typedef struct {
  int32_t n_cams, n_pts;
  int64_t n_obs;
  const double* cam_qt;
  const double* pts;
  const int32_t* obs_cam;
  const int32_t* obs_pt;
  const double* obs_uv;
  const uint8_t* cam_fixed; /* NULL: camera 0 fixed */
  ba_intrinsics K;
  double* cam_qt_out;
  double* pts_out;
} ba_problem;

typedef struct {
  int32_t status;
  int32_t n_iters;
  int32_t n_accepted;
  int32_t pad;
  double initial_cost;
  double final_cost;
  double rmse_px;
  double latency_ms;   /* served: submit -> result available on the host   */
  double cost[BA_MAX_ITERS + 1];
} ba_result;

/* Solve n independent problems with the handle's options (dense solver per
 * problem, max_lm_iters each) in one persistent launch: every CTA takes the
 * next problem from a device work queue and runs its whole LM loop.
 * results[n] receives each problem's costs.  Problems of the batch share
 * nothing, so a result does not depend on the rest of the batch.  The
 * inputs are copied to the device in a compact form: each observation's
 * camera and point in one 32-bit word and, with precision BA_FP32, its
 * pixels rounded to FP32 (the kernels compute in FP32 on that path anyway),
 * so pixel coordinates beyond the FP32 range are refused as non-finite.
 * Errors: INVALID_ARG (a problem fails validation; results[i].status says
 * which), OOM, TIMEOUT, CUDA. */
ba_status ba_solve_batch(ba_handle* h, int32_t n, const ba_problem* problems,
                         ba_result* results);

/* Tile schedule of the batched kernel, as chosen by the autotuner
 * (threads per CTA, CTAs per SM).  ba_tune_batch times candidate schedules
 * on the given problems and keeps the fastest on the handle. */
ba_status ba_get_batch_schedule(const ba_handle* h, int32_t* threads, int32_t* ctas_per_sm);
ba_status ba_set_batch_schedule(ba_handle* h, int32_t threads, int32_t ctas_per_sm);
ba_status ba_tune_batch(ba_handle* h, int32_t n, const ba_problem* problems,
                        int32_t* best_threads, int32_t* best_ctas_per_sm);

/* Create a serving handle: a persistent device worker that admits requests
 * into slots of a device arena as slots and memory free up, runs several at
 * once, and keeps each request's poses, points and LM state resident until
 * it is polled.  opts->serve_* size the arena, slots and queue. */
ba_status ba_create_server(const ba_options* opts, ba_handle** out);

/* Queue one request (copied in; the caller may free its arrays on return).
 * *req_id receives its id.  A request waits on the host when no slot or
 * arena space is free and is admitted as soon as there is.  Errors:
 * INVALID_ARG (validation), BUSY (waiting queue full), STATE (not a server
 * handle), OOM (larger than the whole arena). */
ba_status ba_submit(ba_handle* server, const ba_problem* req, uint64_t* req_id);

/* Collect a request: NOT_READY while it is queued or running; BA_OK once
 * done, with *out filled and the outputs copied into req->cam_qt_out /
 * pts_out as given at submit.  A request is returned once; later polls of
 * the same id give INVALID_ARG. */
ba_status ba_poll(ba_handle* server, uint64_t req_id, ba_result* out);

#ifdef __cplusplus
}
#endif

#endif /* BA_H */
