/*
 * pcg.h -- C-ABI of the GB300 matrix-free line-preconditioned CG solver.
 *
 * The library solves A u = b for the finite-volume discretisation of the
 * anisotropic elliptic model equation of Mueller, Guo, Scheichl, Shi,
 * "Matrix-free GPU implementation of a preconditioned conjugate gradient
 * solver for anisotropic elliptic PDEs" (Section 3, Eq. (ModelEquation)), in
 * the generalised form
 *
 *     -div_h(alpha grad_h u) - (1/S) d_z(S beta d_z u) + lambda^2 u = f
 *
 * on a tensor-product column grid: a periodic rectangle (S = 1), a
 * latitude-longitude band of a spherical shell (S = r^2, Neumann at the
 * latitude edges) or one panel of a gnomonic cubed sphere (the paper's grid,
 * S = r^2, Neumann at the panel edges), with Neumann conditions at the bottom
 * and top of every column.  The operator is never stored: each application recomputes the
 * stencil from per-level profiles and per-column metric terms (Section 4.2).
 * The preconditioner is the vertical-line (block-Jacobi) preconditioner
 * M = block-diag(A), one tridiagonal solve per column (Section 4.2).  The
 * solver is the interleaved PCG loop of Algorithm 1 (Section 4.3) with its
 * two fused grid sweeps (Algorithms 2 and 3 of the appendix).
 *
 * Conventions for every entry point
 * ---------------------------------
 *  - Vectors are contiguous arrays in the layout [nrhs][n_z][n_y][n_x]
 *    (x fastest; each vertical level is one contiguous horizontal plane).
 *  - "Device pointer" arguments are CUDA device (or managed) memory owned by
 *    the caller; the library never frees them.  "Host" arguments are read
 *    during the call and copied; the library keeps no reference to them.
 *  - Work is enqueued on the stream given in pcg_opts_t at creation.  Calls
 *    return after enqueueing unless stated otherwise; stats are final once
 *    the call that fills them has returned.
 *  - Every function returns a pcg_status value; on failure the reason is
 *    available from pcg_last_error().  No function aborts, throws or traps.
 *  - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef PCG_GB300_H
#define PCG_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
enum pcg_status {
    PCG_OK = 0,
    PCG_ERR_INVALID_ARG = 1,   /* bad pointer, size, geometry or option          */
    PCG_ERR_OOM = 2,           /* device or pinned host allocation failed        */
    PCG_ERR_CUDA = 3,          /* a CUDA runtime call failed (text in last_error) */
    PCG_NOT_CONVERGED = 4,     /* maxit reached before the stopping test passed  */
    PCG_BREAKDOWN = 5,         /* <p,Ap> <= 0, <r,z> < 0 or a non-finite scalar    */
    PCG_TIMEOUT = 6,           /* a bounded device-side wait (staged copies of a sweep) gave up; the solve stopped */
    PCG_PENDING = 7            /* pcg_serve_poll: the request has not finished yet */
};

/* ---- geometry / precision selectors ------------------------------------- */
enum pcg_geometry {
    PCG_GEOM_BOX = 0,          /* periodic lx x ly rectangle, heights z_iface    */
    PCG_GEOM_LATLON = 1,       /* lon periodic over 2 pi, lat in [lat0, lat1]    */
    PCG_GEOM_CUBED_PANEL = 2   /* one panel of an equidistant gnomonic cubed sphere (Section 3.2):
                                  tangent coordinates [-1,1]^2, radii z_iface, Neumann panel edges */
};
enum pcg_precision {
    PCG_FP64 = 0,              /* FP64 storage and arithmetic throughout          */
    PCG_MIXED = 1              /* FP32 inner PCG inside FP64 iterative refinement */
};
enum pcg_preconditioner {
    PCG_PREC_LINE = 0,         /* vertical-line preconditioner M = block-diag(A) (Section 4.2) */
    PCG_PREC_MULTIGRID = 1,    /* one V-cycle of geometric multigrid with vertical line smoothing (the
                                  solver Section 8 names as the next step): n_x, n_y halved per level
                                  while both are even, the vertical grid kept; each level the same
                                  discretisation (alpha on a coarse face = mean of its two fine faces);
                                  restriction = sum of the four fine cells, prolongation = its
                                  transpose; one damped (omega = 0.8) block-Jacobi sweep before and
                                  after the coarse correction; coarsest level: its column block
                                  (with one refinement step) if it is one column, else 8 smoothing
                                  sweeps.  PCG_FP64 only. */
    PCG_PREC_MULTIGRID_F32 = 2 /* the same V-cycle computed in FP32 (r rounded to FP32 on the way in, z
                                  widened on the way out) inside the FP64 CG.  PCG_FP64 only. */
};

/* How an iteration is organised on the device (pcg_opts_t.algorithm). */
enum pcg_algorithm {
    PCG_ALG_INTERLEAVED = 0,      /* Algorithm 1 of the paper: a preconditioner sweep and an SpMV sweep per
                                     iteration, two grid-wide reductions */
    PCG_ALG_SINGLE_REDUCTION = 1  /* the Chronopoulos-Gear rearrangement cited in Section 4.3: one sweep and one
                                     reduction per iteration, the line solves of each tile's ring of neighbouring
                                     columns recomputed by the tile.  With PCG_FP64 it is the whole solve, with
                                     PCG_MIXED the FP32 inner solve.  PCG_PREC_LINE and n_z <= 256 only; other
                                     combinations are rejected with PCG_ERR_INVALID_ARG.  x is current when the
                                     stopping test fires. */
};

typedef struct pcg_ctx* pcg_t;
typedef struct pcg_server* pcg_server_t;

/* Grid (Section 3.1: tensor product of a horizontal grid and a graded
 * vertical grid).  z_iface: host array of n_z+1 strictly increasing
 * interface heights (box) or radii (latlon). */
typedef struct {
    int geometry;              /* pcg_geometry                                    */
    int n_x, n_y, n_z;         /* cells per direction, each >= 1                  */
    int nrhs;                  /* right-hand sides solved together, >= 1          */
    const double* z_iface;     /* host, n_z + 1 values                            */
    double lx, ly;             /* box: periodic extents (> 0)                     */
    double lat0, lat1;         /* latlon: band edges in radians, -pi/2 < lat0 < lat1 < pi/2 */
} pcg_grid_t;

/* Coefficients of the model equation, sampled where the finite-volume scheme
 * needs them: alpha at horizontal face midpoints, beta at level interfaces. */
typedef struct {
    const double* alpha_e;     /* host [n_y][n_x]: alpha on the east face of (i,j), or NULL for alpha = 1 */
    const double* alpha_n;     /* host [n_y][n_x]: alpha on the north face of (i,j), or NULL for alpha = 1;
                                  ignored on the northern edge of a latlon band   */
    const double* beta_iface;  /* host, n_z + 1 values (only interior ones enter) */
    double lambda2;            /* zero-order coefficient, >= 0 (> 0 for an SPD system with periodic x, y) */
} pcg_coeffs_t;

typedef struct {
    int precision;             /* pcg_precision                                   */
    double inner_tol;          /* PCG_MIXED: relative tolerance of each FP32 inner solve; 0 selects 1e-5 */
    int inner_maxit;           /* PCG_MIXED: iteration cap of each inner solve; 0 selects 20000 */
    int max_outer;             /* PCG_MIXED: refinement sweeps cap; 0 selects 16   */
    int passes_per_launch;     /* PCG passes per CUDA-graph launch between convergence polls; 0 selects 16
                                  (4 with a multigrid preconditioner)                                  */
    void* stream;              /* cudaStream_t for all work; NULL = default stream */
    int preconditioner;        /* pcg_preconditioner (PCG_PREC_LINE when opts is NULL) */
    int algorithm;             /* pcg_algorithm (PCG_ALG_INTERLEAVED when opts is NULL) */
} pcg_opts_t;

/* Per-solve statistics.  For nrhs > 1 the scalar fields report the worst
 * right-hand side; per-rhs values are available from pcg_rhs_stats(). */
typedef struct {
    int status;                /* pcg_status of the solve                         */
    int iterations;            /* FP64: CG iterations (updates of u); MIXED: inner iterations summed over sweeps */
    int outer_sweeps;          /* MIXED: refinement sweeps taken; FP64: 0         */
    int stagnated;             /* MIXED: 1 if refinement stopped at the FP64 rounding floor (relres_floor) or
                                  because the FP64 residual stopped falling      */
    double relres_recursive;   /* FP64: ||r_k||/||b|| of the updated residual at exit */
    double relres_true;        /* ||b - A x||/||b|| recomputed in FP64 after exit  */
    double elapsed_ms;         /* wall time of the call on the host               */
    double relres_floor;       /* estimate of ||b - A fl(x)||/||b|| for x rounded to FP64,
                                  sqrt(sum_i ulp(x_i)^2/12 ||A e_i||^2)/||b||: the smallest true
                                  residual an FP64 vector can show for this solution */
} pcg_stats_t;

/* Create a solver for one grid and coefficient set (Section 4.2: the level
 * profiles and column metric terms are computed once here and kept on the
 * device; per-column tridiagonal factors of M are precomputed in FP64).
 * All inputs are copied.  On failure *out is set to NULL.
 * Errors: PCG_ERR_INVALID_ARG, PCG_ERR_OOM, PCG_ERR_CUDA. */
int pcg_create(const pcg_grid_t* grid, const pcg_coeffs_t* coeffs, const pcg_opts_t* opts, pcg_t* out);

/* Solve A x = b for all nrhs right-hand sides (Algorithm 1).
 * b, x: device pointers, FP64, nrhs * n_z * n_y * n_x values; x is the
 * initial guess on entry and the solution on return.  The stopping test
 * is ||r_k|| < tol ||b|| on the recursively updated residual (Algorithm 1);
 * tol = 0 runs exactly maxit iterations.  PCG_MIXED refines in FP64 until
 * ||b - A x|| < tol ||b|| or the FP64 residual stops falling.  Blocks the
 * host until the solve has finished; stats may be NULL.
 * Returns PCG_OK, PCG_NOT_CONVERGED, PCG_BREAKDOWN or an error code. */
int pcg_solve(pcg_t h, const double* b, double* x, double tol, int maxit, pcg_stats_t* stats);

/* As pcg_solve, with b and x in host memory (pinned or pageable): copies b
 * and x to the handle's device buffers, solves, copies x back. */
int pcg_solve_host(pcg_t h, const double* b_host, double* x_host, double tol, int maxit, pcg_stats_t* stats);

/* Statistics of right-hand side `rhs` from the last solve. */
int pcg_rhs_stats(pcg_t h, int rhs, pcg_stats_t* stats);

/* y = A x (Section 4.2 stencil, flux form), FP64 device pointers, nrhs
 * vectors.  x and y must not overlap.  Asynchronous on the handle's stream. */
int pcg_apply_A(pcg_t h, const double* x, double* y);

/* z = M^{-1} r, M = block-diag(A) (Section 4.2; one Thomas solve per
 * column), FP64 device pointers, nrhs vectors; r and z must not overlap.
 * For a handle created with PCG_PREC_MULTIGRID, z = B r: one V-cycle from a
 * zero guess.  Asynchronous on the handle's stream. */
int pcg_precond(pcg_t h, const double* r, double* z);

/* FP32 versions of the two operators (the kernels of the FP32 inner solve
 * of PCG_MIXED), FP32 device pointers.  Asynchronous. */
int pcg_apply_A_f32(pcg_t h, const float* x, float* y);
int pcg_precond_f32(pcg_t h, const float* r, float* z);

/* Benchmark helper: starting from x0 = 0 on right-hand side b (FP64 device
 * pointer), run `passes` passes of Algorithm 1 in the FP64 sweeps
 * (precision = PCG_FP64) or the FP32 inner sweeps (PCG_MIXED), launching each
 * sweep on its own between CUDA events on the handle's stream, and return
 * the mean device time per launch of the preconditioner sweep (Algorithm 3)
 * and of the SpMV sweep (Algorithm 2) in milliseconds.  Uses the handle's
 * workspace; blocks until done.  Errors: PCG_ERR_INVALID_ARG, PCG_ERR_CUDA. */
int pcg_time_sweeps(pcg_t h, const double* b, int precision, int passes, double* ms_prec, double* ms_spmv);

/* Benchmark helper: as pcg_time_sweeps, but the `passes` passes run back to
 * back as in a solve (no event between the sweeps; the FP32 sweeps of
 * PCG_MIXED overlap their neighbours' start and end as in the solve's
 * graphs), and the mean device time of one pass (preconditioner sweep plus
 * SpMV sweep) is returned in *ms_per_pass.  Blocks until done.  Errors:
 * PCG_ERR_INVALID_ARG, PCG_ERR_CUDA. */
int pcg_time_passes(pcg_t h, const double* b, int precision, int passes, double* ms_per_pass);

/* z = M^{-1} r like pcg_precond, for a caller that must not allocate device
 * memory when it calls: a real-time loop that cannot take the latency (or the
 * implicit synchronisation) of a cudaMalloc, or a host whose device memory
 * all belongs to another allocator (a framework's caching allocator, a fixed
 * budget), where a library-side cudaMalloc would fail or fragment it.  Such a
 * caller cannot create a handle at that point, since pcg_create allocates.
 * There is no counterpart in the paper; it exists for those callers.
 * Nothing is allocated: the operator tables and Thomas factors go into one
 * fixed 4 MiB device array owned by the library (every GPU that loads the
 * library holds it until exit), so the grid must satisfy
 *     3 n_z + a + 2 n_x n_y + 3 n_z c <= 524288,
 * a = n_y (box, latlon) or n_x n_y (cubed panel), c = 1 (box, alpha NULL),
 * n_y (latlon, alpha NULL) or n_x n_y (alpha given, or the cubed panel);
 * larger grids return PCG_ERR_INVALID_ARG with the sizes in
 * pcg_last_error(NULL).  grid, coeffs: host descriptions as for pcg_create,
 * any of the three geometries (read during the call); r, z: FP64 device
 * pointers, nrhs vectors, not overlapping.  stream: cudaStream_t (NULL =
 * default stream).  The tables are computed on the host into one static host
 * buffer of the library and copied to the device array by cudaMemcpyAsync on
 * `stream` (a copy from pageable memory returns once the buffer has been
 * read); the factor and solve kernels follow on the same stream.  The first
 * call on each device looks up the array's device address (with that device
 * current); make that first call before any stream capture begins on the
 * device.  Every call rewrites the whole array and the staging buffer, so
 * calls whose work overlaps on the GPU (other streams) race on the array, and
 * calls from several host threads at once race on the staging buffer.
 * Errors: PCG_ERR_INVALID_ARG, PCG_ERR_CUDA (text in pcg_last_error(NULL)). */
int pcg_precond_noalloc(const pcg_grid_t* grid, const pcg_coeffs_t* coeffs, const double* r, double* z, void* stream);

/* ---- served batch (continuous batching of many solves) ------------------ */

/* Create a server that solves many independent problems of different grids,
 * coefficients and right-hand sides together.  budget_bytes bounds the
 * device memory of admitted requests; max_slots bounds how many are admitted
 * at once (<= 4096).  opts (may be NULL) selects one of two modes by
 * opts->preconditioner:
 *  - PCG_PREC_LINE (default): the mixed-precision form (FP32 inner
 *    Algorithm 1 inside FP64 refinement, as pcg_solve with PCG_MIXED), the
 *    inner iterations of all admitted requests advancing together in
 *    persistent batched sweeps; about 36 bytes per unknown (tables, FP64 x
 *    and b, five FP32 inner vectors).  inner_tol, inner_maxit, max_outer as
 *    for pcg_create; passes_per_launch = epochs per CUDA-graph launch
 *    (default 8); stream = the stream of the batched work.
 *  - PCG_PREC_MULTIGRID_F32: FP64 CG preconditioned by the FP32 V-cycle (as
 *    pcg_solve on a handle created with it), each request on a handle of its
 *    own, solved by one of min(max_slots, 16) worker threads with a stream
 *    each, so up to that many solves run at once and overlap on the device;
 *    a solve is restarted from x until the true residual is below tol or
 *    within twice the FP64 rounding floor (at most four solves;
 *    stats.outer_sweeps counts them).  About 96 bytes per unknown.
 * Other preconditioner values return PCG_ERR_INVALID_ARG.
 * Errors: PCG_ERR_INVALID_ARG, PCG_ERR_OOM, PCG_ERR_CUDA. */
int pcg_server_create(size_t budget_bytes, int max_slots, const pcg_opts_t* opts, pcg_server_t* out);

/* Queue one solve (nrhs must be 1).  grid, coeffs, b_host (n_z*n_y*n_x
 * values, layout as everywhere) are copied; tol as for pcg_solve with
 * PCG_MIXED.  The request is admitted when a slot and the byte budget allow
 * (first in, first out): by a later pcg_serve_step in the batched mode, by a
 * free worker in the multigrid mode.  A request larger than
 * the whole budget fails here with PCG_ERR_OOM; invalid geometry with
 * PCG_ERR_INVALID_ARG.  *req_id identifies the request. */
int pcg_serve_submit(pcg_server_t s, const pcg_grid_t* grid, const pcg_coeffs_t* coeffs, const double* b_host,
                     double tol, uint64_t* req_id);

/* Multigrid mode: the workers advance on their own; pcg_serve_step waits
 * at most a millisecond for a request to finish and reports the counts.
 * Batched mode: advance the served batch: admit waiting requests, run the FP64
 * refinement steps that are due, and run inner PCG epochs (one epoch = one
 * pass of Algorithm 1 for every request in its inner phase, executed by
 * persistent kernels over the work list of (request, 32x4-column tile)
 * items) until at least max_epochs epochs have run or no request has inner
 * work; requests that finish are retired and their memory returned.
 * Blocks the host.  *n_active / *n_pending (may be NULL): requests admitted /
 * still queued afterwards. */
int pcg_serve_step(pcg_server_t s, int max_epochs, int* n_active, int* n_pending);

/* PCG_PENDING while request req_id is unfinished; once finished, copies x
 * (host, n_z*n_y*n_x values; may be NULL) and the statistics (elapsed_ms =
 * submission to retirement) and returns PCG_OK, after which the id is
 * forgotten.  The request's own outcome is stats->status. */
int pcg_serve_poll(pcg_server_t s, uint64_t req_id, double* x_host, pcg_stats_t* stats);

/* Counters of the server: admitted and queued requests, device bytes held
 * by admitted requests, inner epochs run so far.  Any pointer may be NULL. */
int pcg_serve_info(pcg_server_t s, int* n_active, int* n_pending, size_t* used_bytes, long long* epochs);

/* Text of the last error of the server (or of the last failed
 * pcg_server_create on this thread when s is NULL). */
const char* pcg_server_last_error(pcg_server_t s);

/* Free all device and host memory of the server, finished or not (in the
 * multigrid mode after the solves in flight have finished). */
void pcg_server_destroy(pcg_server_t s);

/* Block the host until all work enqueued on the handle's stream is done. */
int pcg_sync(pcg_t h);

/* Device bytes held by the handle (workspace and tables). */
size_t pcg_device_bytes(pcg_t h);

/* Number of kernels the last solve launched (graph nodes included). */
long long pcg_kernel_launches(pcg_t h);

/* Text of the last error on this handle (or of the last failed pcg_create
 * on this thread when h is NULL).  Never NULL. */
const char* pcg_last_error(pcg_t h);

/* Free everything the handle allocated; caller buffers are untouched. */
void pcg_destroy(pcg_t h);

#ifdef __cplusplus
}
#endif
#endif /* PCG_GB300_H */
