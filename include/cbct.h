/*
 * cbct.h -- C ABI of the GB300 cone-beam CT reconstruction library (libcbct.so).
 *
 * The library computes the two matrix-vector products every Krylov method of
 * Sabate Landman, Biguri et al., "On Krylov Methods for Large Scale CBCT
 * Reconstruction", spends its time on (Sec. 2: one product with A and one with
 * A^T make up almost all of an iteration's cost):
 *
 *   y = A x     forward projection, A in R^{N x M} (Sec. 1, Eq. 1),
 *   x = A^T y   its exact transpose (backprojection),
 *
 * and the solvers of Sec. 2.1-2.2 built around them, with every vector kept on
 * the GPU and every Krylov scalar in FP64.
 *
 * System matrix.  A[i][j] is the length (mm) of ray i inside voxel j.  Ray i
 * is the segment from the X-ray source to the centre of detector pixel i;
 * voxel j is a half-open box.  N = nangles * nv * nu rays, M = nx * ny * nz.
 *
 * Geometry conventions (the paper leaves them to its toolbox):
 *   rotation axis = z, origin = rotation centre = volume centre;
 *   source at (dso cos t, dso sin t, 0) for source angle t;
 *   detector centre at -(dsd - dso) (cos t, sin t, 0);
 *   detector axes e_u = (-sin t, cos t, 0), e_v = (0, 0, 1);
 *   pixel (iu, iv) centre = detector centre + (iu - (nu-1)/2) du e_u
 *                                          + (iv - (nv-1)/2) dv e_v;
 *   voxel (i, j, k) = [x0 + i dx, x0 + (i+1) dx) x [...] x [...],
 *                     x0 = -nx dx / 2 (likewise y, z).
 * Layout: volumes are x[k][j][i] (x fastest), projection stacks are
 * y[a][iv][iu] (u fastest), both dense and row-major.
 *
 * Threading and streams.  Every call that takes a stream enqueues its GPU work
 * on that stream (NULL = the legacy default stream).  Solvers synchronise the
 * stream once at the end to copy their report to the host.  A geometry may be
 * shared by calls on different streams and host threads.
 *
 * Errors.  Every call returns a cbct_status; nothing is thrown across the ABI.
 * cbct_last_error() returns a message for the calling thread's last failure.
 */
#ifndef CBCT_H
#define CBCT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (binary-compatible with cudaStream_t); NULL = default stream. */
typedef struct CUstream_st *cbct_stream;

typedef enum {
    CBCT_OK = 0,
    CBCT_EINVAL = 1,      /* bad argument: null pointer, size, non-physical geometry */
    CBCT_ENOMEM = 2,      /* device or host allocation failed */
    CBCT_ECUDA = 3,       /* a CUDA runtime call failed (message has the CUDA error) */
    CBCT_EBREAKDOWN = 4,  /* a Krylov scalar became zero or non-finite; x holds the last finite iterate */
    CBCT_ETIMEOUT = 5,    /* a bounded wait gave up (serving) */
    CBCT_EBUDGET = 6,     /* request larger than the serving HBM budget */
    CBCT_ENOTFOUND = 7    /* unknown request id (serving) */
} cbct_status;

/* Storage type of volumes / projections / Krylov vectors.  Arithmetic is FP32
 * (projectors) and FP64 (Krylov scalars) whatever the storage type. */
typedef enum { CBCT_F32 = 0, CBCT_F16 = 1, CBCT_BF16 = 2 } cbct_dtype;

/* Circular cone-beam scan.  Lengths in mm, angles in radians.  Requirements:
 * all counts >= 1, all sizes > 0, dsd > dso, and the source and detector must
 * lie outside the cylinder that circumscribes the volume. */
typedef struct {
    int nx, ny, nz;               /* voxels */
    double dx, dy, dz;            /* voxel size */
    int nu, nv;                   /* detector pixels (u = in-plane, v = axial) */
    double du, dv;                /* pixel pitch */
    double dso, dsd;              /* source-origin and source-detector distances */
    int nangles;                  /* projections */
    const double *angles_rad;     /* host array of nangles source angles; copied */
} cbct_geometry_desc;

typedef struct cbct_geometry cbct_geometry;   /* opaque, library-owned */

/* Builds the device-side ray tables of a scan (on the current CUDA device).
 * On success *out owns device memory until cbct_geometry_destroy.  Every
 * call below that queues GPU work for a geometry must be made with the
 * geometry's device current; otherwise it returns CBCT_EINVAL before any
 * work is queued (the caller's buffers must live on that device too). */
cbct_status cbct_geometry_create(const cbct_geometry_desc *desc, cbct_geometry **out);
void cbct_geometry_destroy(cbct_geometry *geom);
/* Ordinal of the CUDA device the geometry's tables live on, or -1 for NULL. */
int cbct_geometry_device(const cbct_geometry *geom);
int64_t cbct_geometry_num_voxels(const cbct_geometry *geom);   /* M, or -1 for NULL */
int64_t cbct_geometry_num_rays(const cbct_geometry *geom);     /* N, or -1 for NULL */

/* y = A x (Sec. 1, Eq. 1).  x: M device elements, y: N device elements, both
 * of `dtype`, caller-owned, non-overlapping.  Ray sums are FP32 (Kahan-
 * compensated for F16/BF16 storage).  Asynchronous on `stream`. */
cbct_status cbct_project(const cbct_geometry *geom, const void *x, void *y,
                         cbct_dtype dtype, cbct_stream stream);

/* x = A^T y, the transpose of cbct_project (the same ray/voxel lengths from
 * the same crossing tables, so <A x, y> = <x, A^T y> up to FP32 rounding of
 * the lengths and sums; Sec. 2.1.4 explains why an unmatched backprojector
 * breaks the Krylov methods).  y: N device
 * elements, x: M device elements of `dtype`.  Asynchronous on `stream`. */
cbct_status cbct_backproject(const cbct_geometry *geom, const void *y, void *x,
                             cbct_dtype dtype, cbct_stream stream);

/* cbct_project without any device allocation, for callers that cannot call
 * cudaMalloc (the paper has no counterpart: it is an interface variant, not a
 * step of the method).  Same arguments, layouts and result as cbct_project;
 * the padded z-fastest copy of the volume (nx * ny * (nz + 2) + 4 elements)
 * that cbct_project allocates per call lives here in a fixed 66 MiB array of
 * the library's device memory, so e.g. a 256^3 FP32 volume or a 256^2 x 512
 * FP16/BF16 volume fits; larger ones are rejected with CBCT_EINVAL before any
 * work is queued.  The geometry's device must be the current device (else
 * CBCT_EINVAL).  The first call on a device looks the array up
 * (cudaGetSymbolAddress); make it before capturing a stream.  Every call on a
 * device shares the one array, which keeps the last call's contents (each
 * call overwrites all it reads): calls whose work overlaps on the GPU (other
 * streams, other threads) race and give wrong results, so serialise them on
 * one stream. */
cbct_status cbct_project_static(const cbct_geometry *geom, const void *x, void *y,
                                cbct_dtype dtype, cbct_stream stream);

/* A voxel-driven, interpolating backprojector: an approximation of A^T that is
 * not its transpose, the kind of backprojector Sec. 2.1.4 says fast CBCT codes
 * use.  Every voxel centre is projected onto every detector, the projection
 * is sampled there by bilinear interpolation (zero outside the detector) and
 * weighted by dx dy dz mag^2 |d'| / (du dv DSD), the expected sum of A's
 * entries of the rays through the voxel (mag = DSD / (DSO - <c, s_hat>), |d'|
 * the source-to-sample distance).  y: N FP32 device values y[a][iv][iu];
 * x: M FP32 device values x[k][j][i].  Asynchronous on `stream`. */
cbct_status cbct_backproject_voxel_driven(const cbct_geometry *geom, const float *y, float *x,
                                          cbct_stream stream);

/* Number of nonzeros of A (positive-length ray/voxel pairs in FP32), counted
 * by the forward traversal.  Synchronises `stream`. */
cbct_status cbct_count_nnz(const cbct_geometry *geom, int64_t *nnz, cbct_stream stream);

/* Launch shapes of the projectors of one geometry (performance only: every
 * shape computes the same A and A^T).  fwd_rows: rays per lane of the forward
 * tile (1, 2 or 4; a warp follows 32 * fwd_rows rows of one detector column).
 * bwd_config: tile of the transpose (one warp per voxel column), 0 = 4 x 2
 * columns x 32 voxels along z (1 per lane), 1 = 4 x 2 x 64 (2 per lane),
 * 2 = 8 x 1 x 32, 3 = 2 x 4 x 64, 4 = 4 x 2 x 128 (4 per lane),
 * 5 = 2 x 4 x 128, 6 = 4 x 2 x 256 (8 per lane), 7 = 2 x 4 x 256,
 * 8 = 2 x 4 x 128 and 9 = 4 x 2 x 128 holding each voxel's candidate rows in
 * registers per angle (configurations 0..3 do too; 4..7 re-read them per
 * detector column).  Changing the shape while another thread uses the
 * geometry is a data race. */
#define CBCT_TUNE_TIMES 13
cbct_status cbct_geometry_set_launch(cbct_geometry *geom, int fwd_rows, int bwd_config);
cbct_status cbct_geometry_get_launch(const cbct_geometry *geom, int *fwd_rows, int *bwd_config);
/* Times every launch shape (forward and transpose, FP32, on a strided subset
 * of at most max_angles angles; max_angles <= 0 = all) and keeps the fastest.
 * The subset is widened to at least twice the device's L2 size worth of
 * projections (or all angles), so that the transpose is timed reading its
 * projections from HBM as in a full-size product, not from L2.
 * times_ms, if non-null, is a host array of CBCT_TUNE_TIMES doubles that
 * receives the forward times for fwd_rows 1, 2, 4 and the transpose times for
 * bwd_config 0..9.  Allocates scratch on `stream` and synchronises it. */
cbct_status cbct_geometry_autotune(cbct_geometry *geom, int max_angles, double *times_ms, cbct_stream stream);
/* Angles per pass of the transpose inside the solvers and cbct_backproject
 * (performance only).  With a
 * projection stack larger than L2 the transpose runs in passes over blocks of
 * `angles` consecutive angles, keeping FP32 running sums in M values of
 * scratch, so that each pass gathers from projections that stay in L2.
 * angles >= nangles means one pass; angles == 0 restores the default (one
 * pass); negative values are rejected (CBCT_EINVAL).  Every block size gives
 * bit-identical sums (the running sums are kept in FP32 between passes, in
 * the same order).  Not thread-safe, like set_launch. */
cbct_status cbct_geometry_set_angle_block(cbct_geometry *geom, int angles);
cbct_status cbct_geometry_get_angle_block(const cbct_geometry *geom, int *angles);

/* ------------------------------------------------------------------ solvers
 * All solvers start from x_0 = 0 and run opts->iters iterations (fewer on
 * breakdown).  b (N FP32 values) and x (M FP32 values, output only) may be
 * device or host pointers; host buffers are staged through device memory.
 * Each iteration applies A once and A^T once; the loop runs without host
 * synchronisation (optionally replayed as a CUDA graph).  The library
 * allocates its workspace per call with stream-ordered allocation and frees
 * it before returning. */

typedef enum { CBCT_LAMBDA_FIXED = 0, CBCT_LAMBDA_GCV = 1, CBCT_LAMBDA_DP = 2 } cbct_lambda_rule;

typedef struct {
    int iters;               /* iterations (>= 1) */
    double lambda;           /* Tikhonov lambda (Sec. 2.2, Eq. 6): damping of CGLS/LSQR/LSMR,
                                or the fixed lambda of hybrid LSQR with CBCT_LAMBDA_FIXED */
    cbct_lambda_rule rule;   /* hybrid LSQR only: fixed lambda, GCV or the discrepancy
                                principle (Sec. 2.2.2) */
    cbct_dtype storage;      /* storage type of the Krylov vectors (u, v, basis V_k) */
    int use_graph;           /* nonzero: capture one iteration as a CUDA graph and replay it */
    int profile;             /* nonzero: time every projector launch with CUDA events (disables
                                the graph) and fill the report's *_ms fields */
    double noise_level;      /* CBCT_LAMBDA_DP: nl = ||e|| / ||b||; lambda_k is the root of
                                ||b - A x_lambda|| = nl ||b|| on the projected problem, found by
                                bisection in log lambda over sigma_max [1e-8, 1e8]; 0 while even
                                the smallest lambda leaves the residual above the target */
    int explicit_residual;   /* nonzero: after every iteration compute ||b - A x_k|| with one more
                                forward projection and stop at the first k where it exceeds
                                (1 - stop_tol) times the previous one, returning x_{k-1} (the
                                paper's toolbox stops once the explicit residual increases,
                                Sec. 3.1.1); costs one product with A per iteration */
    double stop_tol;         /* 0 <= stop_tol < 1; 0 = stop on increase */
    int gmres_backprojector; /* AB-/BA-GMRES: 0 = B = A^T; 1 = B = C A^T R with the SIRT weights
                                R = 1 / (A 1), C = 1 / (A^T 1); 2 = the voxel-driven
                                interpolating backprojector (cbct_backproject_voxel_driven);
                                1 and 2 are not the transpose of A */
    int tv_outer;            /* CGLS-TV: reweighting (outer) steps, 1 <= tv_outer <= iters; the
                                iters CGLS iterations are spread evenly over them */
    double tv_tau;           /* CGLS-TV: smoothing tau > 0 of the weights (|D x|^2 + tau^2)^(-1/4) */
    int reorth;              /* LSQR, LSMR, hybrid LSQR/LSMR: nonzero = re-orthogonalise every new
                                u and v against all earlier ones (classical Gram-Schmidt twice,
                                FP64 dots; Sec. 3.1.1 and Sec. 4), keeping (iters + 1) normalised
                                vectors of each kind; FP32 storage only */
} cbct_solve_opts;

/* Per-iteration histories, written to caller-allocated HOST arrays of length
 * >= opts->iters (any pointer may be NULL).  resid_norm: the solver's estimate
 * of ||b - A x_k|| (of the damped residual when lambda > 0); normal_resid_norm:
 * its estimate of ||A^T (b - A x_k) - lambda^2 x_k||; lambda_k: hybrid LSQR's
 * lambda per iteration. */
typedef struct {
    int iters_done;
    double *resid_norm;
    double *normal_resid_norm;
    double *lambda_k;
    int64_t kernel_launches;     /* out: kernels this call launched (graph replays count each node) */
    int64_t forward_launches;    /* out: forward-projector launches */
    int64_t backward_launches;   /* out: backprojector launches */
    double forward_ms;           /* out, profile != 0: summed device time of the forward launches */
    double backward_ms;          /* out, profile != 0: summed device time of the backprojector launches */
    double *explicit_resid_norm; /* explicit_residual: ||b - A x_k|| per completed iteration, plus the
                                    one that triggered the stop (host array of length >= iters) */
    int explicit_count;          /* out: entries written to explicit_resid_norm */
    int stopped_on_residual;     /* out: 1 if the explicit-residual rule ended the solve; the
                                    returned x is then x_{iters_done}, iters_done = count - 1 */
} cbct_solve_report;

/* CGLS (Sec. 2.1.1, Eq. 3). */
cbct_status cbct_cgls_solve(const cbct_geometry *geom, const float *b, float *x,
                            const cbct_solve_opts *opts, cbct_solve_report *report,
                            cbct_stream stream);
/* LSQR (Sec. 2.1.2, Eq. 4): Golub-Kahan bidiagonalisation + Paige-Saunders recurrences. */
cbct_status cbct_lsqr_solve(const cbct_geometry *geom, const float *b, float *x,
                            const cbct_solve_opts *opts, cbct_solve_report *report,
                            cbct_stream stream);
/* LSMR (Sec. 2.1.3, Eq. 5; damped form of Sec. 2.2, Eq. 7 when lambda > 0). */
cbct_status cbct_lsmr_solve(const cbct_geometry *geom, const float *b, float *x,
                            const cbct_solve_opts *opts, cbct_solve_report *report,
                            cbct_stream stream);
/* Hybrid LSQR (Sec. 2.2.1, Eq. 8): Tikhonov on the projected problem with
 * lambda_k fixed or chosen by GCV (Sec. 2.2.2).  Keeps the basis V_k on the
 * device (iters + 1 volumes of the storage type). */
cbct_status cbct_hybrid_lsqr_solve(const cbct_geometry *geom, const float *b, float *x,
                                   const cbct_solve_opts *opts, cbct_solve_report *report,
                                   cbct_stream stream);
/* CGLS-TV (Sec. 2.3.1): isotropic 3D total variation by iteratively
 * reweighted norms.  Each of the tv_outer steps fixes the weights
 * W = diag((|D x|^2 + tv_tau^2)^(-1/4)) from the current x (uniform at x_0 = 0)
 * and runs CGLS on min ||A x - b||^2 + lambda^2 ||W D x||^2 from the current x,
 * with D the forward-difference gradient (zero last difference, Neumann
 * boundary) along i, j, k; lambda is opts->lambda.  resid_norm receives
 * ||b - A x|| and normal_resid_norm the stacked system's normal residual after
 * every CGLS iteration; an outer step ends early once that normal residual
 * falls to 1e-14 of its start.  FP32 storage only. */
cbct_status cbct_cgls_tv_solve(const cbct_geometry *geom, const float *b, float *x,
                               const cbct_solve_opts *opts, cbct_solve_report *report, cbct_stream stream);

/* AB-GMRES and BA-GMRES (Sec. 2.1.4): GMRES with the backprojector B as a
 * right or left preconditioner, for backprojectors that are not exactly the
 * transpose of A.  AB: x_k = B z_k with z_k minimising ||b - A B z|| over
 * K_k(A B, b); BA: x_k minimises ||B (b - A x)|| over K_k(B A, B b).  B is set
 * by opts->gmres_backprojector; with B = A^T they reach LSQR's (AB) and LSMR's
 * (BA) iterates in exact arithmetic.  Arnoldi with classical Gram-Schmidt
 * applied twice (FP64 dots), FP32 Krylov vectors ((iters + 1) of them, rays
 * for AB, voxels for BA), the Hessenberg least-squares problem in FP64.
 * resid_norm (AB) or normal_resid_norm (BA) receive the minimised residual per
 * iteration; iters_done is smaller than iters if the Krylov space is
 * exhausted.  FP32 storage only; the explicit-residual monitor is rejected. */
cbct_status cbct_ab_gmres_solve(const cbct_geometry *geom, const float *b, float *x,
                                const cbct_solve_opts *opts, cbct_solve_report *report, cbct_stream stream);
cbct_status cbct_ba_gmres_solve(const cbct_geometry *geom, const float *b, float *x,
                                const cbct_solve_opts *opts, cbct_solve_report *report, cbct_stream stream);

/* Hybrid LSMR: the extension of the hybrid method to LSMR that Sec. 2.2.2
 * mentions (LSMR's own projected system in place of LSQR's): Tikhonov on
 * LSMR's projected problem, y_k = argmin ||alpha_1 beta_1 e_1 - Hbar_k y||^2 +
 * lambda_k^2 ||y||^2 with Hbar_k = [H_k^T H_k ; alpha_{k+1} beta_{k+1} e_k^T],
 * x_k = V_k y_k (x_k minimises ||A^T (b - A x)||^2 + lambda_k^2 ||x||^2 over
 * the Krylov space).  lambda_k fixed or by GCV on that problem
 * (CBCT_LAMBDA_DP is rejected: it bounds ||r||, not ||A^T r||);
 * normal_resid_norm receives ||alpha_1 beta_1 e_1 - Hbar_k y_k||. */
cbct_status cbct_hybrid_lsmr_solve(const cbct_geometry *geom, const float *b, float *x,
                                   const cbct_solve_opts *opts, cbct_solve_report *report,
                                   cbct_stream stream);

/* ------------------------------------------------------------------ serving
 * A server reconstructs many scans concurrently on the current CUDA device
 * ("continuous batching"; no counterpart in the paper, which solves one scan at
 * a time).  Submitted requests wait in FIFO order and are admitted as slots
 * while the device memory they need fits the budget; a library-owned worker
 * thread then runs steps: one Krylov iteration of a set of admitted requests
 * (one multi-instance launch per kernel for all of them).  Two more library
 * threads keep host-side work off the steps' path: one admits waiting
 * requests (builds the scan's tables, uploads b and queues the solver's start
 * on its own CUDA stream), one reads finished results out to the host and
 * frees their memory.  Which admitted requests a step advances is the
 * schedule.  CBCT_SCHED_FIFO takes them in submission order while the
 * step's forward tiles (8 detector columns x 128 rows of one angle each) stay
 * within 2048, so small requests share a step and large ones run one at a
 * time, oldest first (the order that minimises the longest wait).  A step
 * of one request that fills the GPU alone runs the single-request projector
 * kernels, and under FIFO all of that request's remaining iterations are
 * queued before the worker looks at the device again;
 * CBCT_SCHED_SRPT takes them in order of least remaining work (iterations
 * left x rays x (nx + ny)) under the same limit, which shortens the median
 * latency but makes long requests wait behind short ones (a request left out
 * of 64 consecutive steps goes first from then on, so it cannot starve);
 * CBCT_SCHED_RATIO orders them by response ratio (age + remaining time) /
 * remaining time (remaining time from the same cost model and the measured
 * work rate); CBCT_SCHED_SHARE advances every admitted request every step.
 * Each result equals the single-request solver's up to FP32 rounding: the
 * server's tiles sum every ray and voxel in the same order, but a single
 * request tuned to other launch shapes (cbct_geometry_autotune) sums its norm
 * partials in other groups, and late iterates of ill-conditioned problems
 * amplify such differences (about 1e-4 relative after 20-40 iterations).
 * Requests use FP32 storage and LSQR or LSMR.  All calls are thread-safe
 * except cbct_server_destroy, which must not overlap any other call on the
 * same server. */

typedef struct cbct_server cbct_server;   /* opaque, library-owned */
typedef enum { CBCT_SOLVER_LSQR = 0, CBCT_SOLVER_LSMR = 1 } cbct_solver;

typedef enum { CBCT_SCHED_SRPT = 0, CBCT_SCHED_SHARE = 1, CBCT_SCHED_RATIO = 2, CBCT_SCHED_FIFO = 3 } cbct_schedule;

typedef struct {
    size_t hbm_budget_bytes;   /* device memory the server may hold for requests (> 0) */
    int max_slots;             /* most requests in flight at once (1..64) */
    int use_graph;             /* nonzero: replay each step as one captured CUDA graph */
    int schedule;              /* cbct_schedule: which admitted requests a step advances */
} cbct_server_opts;

typedef struct {
    double submit_s;           /* host steady clock, seconds since the server was created */
    double admit_s;            /* when the request got a slot */
    double finish_s;           /* when its result was on the host */
} cbct_request_times;

/* Starts the worker thread on the current device. */
cbct_status cbct_server_create(const cbct_server_opts *opts, cbct_server **out);
/* Queues a request.  desc: the scan (validated like cbct_geometry_create);
 * b_host: N FP32 measurements on the host, copied before returning; opts:
 * iters >= 1, lambda = Tikhonov damping, storage must be CBCT_F32 (rule,
 * use_graph and profile are ignored).  CBCT_EBUDGET if the request alone
 * needs more than the budget.  *id identifies the request. */
cbct_status cbct_server_submit(cbct_server *srv, const cbct_geometry_desc *desc, const float *b_host,
                               cbct_solver solver, const cbct_solve_opts *opts, uint64_t *id);
/* Device memory a request of this scan, solver and iteration count holds at
 * its peak: what cbct_server_submit charges against the budget (ray tables,
 * Krylov vectors, staging of b, norm partials, state and histories).  Host
 * arithmetic only (no device needed); CBCT_EINVAL on a null pointer, an
 * invalid geometry, a solver other than LSQR / LSMR or iters < 1. */
cbct_status cbct_server_request_bytes(const cbct_geometry_desc *desc, cbct_solver solver, int iters, size_t *bytes);
/* *done = 1 once the request's result is ready (CBCT_ENOTFOUND for unknown ids). */
cbct_status cbct_server_poll(cbct_server *srv, uint64_t id, int *done);
/* Waits up to timeout_s seconds (< 0: forever) for the request.  On time-out
 * returns CBCT_ETIMEOUT and keeps the request.  Otherwise copies the result
 * (M FP32 voxels, x[k][j][i]) into x_host, the histories into report (as for
 * the solvers; may be NULL) and the timestamps into times (may be NULL),
 * forgets the request and returns its status. */
cbct_status cbct_server_wait(cbct_server *srv, uint64_t id, double timeout_s, float *x_host,
                             cbct_solve_report *report, cbct_request_times *times);
/* Counters: steps run, CUDA-graph replays, bytes currently held, requests in slots and waiting.
 * A request is done (and cbct_server_wait returns) as soon as its result is on
 * the host; its device memory is freed right after, so bytes_in_use can lag
 * the last wait by the time of those frees. */
typedef struct {
    int64_t steps, graph_replays;
    size_t bytes_in_use;
    int active, pending;
} cbct_server_stats;
cbct_status cbct_server_get_stats(cbct_server *srv, cbct_server_stats *stats);
/* Stops the worker, drops waiting and active requests and frees everything. */
void cbct_server_destroy(cbct_server *srv);

/* Message describing the calling thread's most recent error ("" if none). */
const char *cbct_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CBCT_H */
