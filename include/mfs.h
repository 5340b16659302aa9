/*
 * mfs.h -- C ABI of the matrix-free first-order conic solver (arXiv 2203.05027) on B300.
 *
 * Problem (Sec. II, eq. prob_primal):   minimize c^T x   subject to  A x = b,  x in K,
 * A in R^{m x n} sparse with o nonzeros, K = K_{n_1} x ... x K_{n_q} a product of cones listed in
 * order over x's coordinates. Two cone kinds: MFS_CONE_NONNEG (a nonnegative orthant of the given
 * size, i.e. that many size-1 Lorentz cones; the LP case of Sec. V) and MFS_CONE_SOC (one Lorentz
 * cone {w : w_1 >= ||w_{2..s}||_2}, Sec. II).
 *
 * Method (Sec. IV, Algorithm 1): two-block ADMM on the UV reformulation A = U V^T (eq. UU/VV),
 * whose x-step (eq. vvt) and y-step (with the matrix inversion lemma) need only the diagonal
 * factors F_V = (I + V V^T)^{-1}, F_U = (I + U U^T)^{-1}. The library runs the equivalent reduced
 * form on n- and m-length vectors (after any iteration gamma = -U^T lambda and
 * y = V^T x + U^T F_U (b - A x)), state (x, z, delta, lambda):
 *     v      = F_U (b - A x_prev) - lambda/mu
 *     x      = F_V ( d .* x_prev + A^T v + z + (delta - c)/mu )      d_j = nonzeros of column j
 *     z      = proj_K(x - delta/mu);   delta += mu (z - x)
 *     lambda -= mu F_U (b - A x)
 * Each iteration is one sweep over A's nonzeros in column order and one in row order.
 *
 * Conventions for every call:
 *  - Every function returns an mfs_status; none aborts or exits. After a failure,
 *    mfs_last_error() gives a one-line reason.
 *  - Input arrays are read, never retained: the library copies them. Output arrays are owned by
 *    the caller and must hold the stated number of elements.
 *  - "host" pointers are ordinary CPU memory; "device" pointers are CUDA device memory of the
 *    device that was current at mfs_create.
 *  - All work is ordered on the CUDA stream given to mfs_create (NULL = legacy default stream).
 *    Calls return after their work has finished, except where a comment says otherwise.
 *  - A solver handle must not be used by two host threads at the same time.
 */
#ifndef MFS_H
#define MFS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mfs_solver mfs_solver; /* opaque; owns all of its device memory */

typedef enum {
    MFS_OK = 0,          /* success; for mfs_solve: the tolerance was reached */
    MFS_MAX_ITER = 1,    /* mfs_solve: max_iter reached before the tolerance */
    MFS_ERR_INVALID = 2, /* bad argument: sizes, indices, cone list, non-finite data, NULL */
    MFS_ERR_CUDA = 3,    /* a CUDA call failed (no device, launch failure, ...) */
    MFS_ERR_OOM = 4,     /* device or host allocation failed */
    MFS_ERR_NUMERIC = 5, /* NaN or Inf in the iterate's residuals */
    MFS_ERR_TIMEOUT = 6, /* a bounded on-device wait gave up; the results of that call are void */
    MFS_INFEASIBLE = 7,  /* mfs_solve: the dual iterates give a certificate that Ax = b, x in K has no solution */
    MFS_UNBOUNDED = 8    /* mfs_solve: the primal iterates give a ray along which c^T x falls without end */
} mfs_status;

enum { MFS_CONE_NONNEG = 0, MFS_CONE_SOC = 1 };

/* Arithmetic of the sweep. MFS_FP64: FP64 storage and arithmetic everywhere.
   MFS_FP32_MIXED: FP32 storage of A, b, c and the iterate and FP32 sweep arithmetic; the residual,
   objective and gap reductions read that data and accumulate in FP64; mfs_solve finishes with
   FP64 iterations (see mfs_settings.polish_iters). */
enum { MFS_FP64 = 0, MFS_FP32_MIXED = 1 };

/* Stopping rule of mfs_solve (mfs_settings.stop_rule); each is "measure <= tol" on a field of
   mfs_residuals_t. MFS_STOP_KKT: the relative KKT residual kkt (the default). MFS_STOP_SCS_L2:
   r_scs, the l2 rule the paper uses against SCS (Sec. V-B). MFS_STOP_OSQP_INF: r_osqp, the
   infinity-norm rule it uses against OSQP (Sec. V-A), without its gap clause, which compares with
   the competing solver's own gap. */
enum { MFS_STOP_KKT = 0, MFS_STOP_SCS_L2 = 1, MFS_STOP_OSQP_INF = 2 };

/* Sweep kernels of the FP32 iteration (mfs_set_sweep). MFS_SWEEP_CHUNKED: one warp per chunk of
   at most 256 nonzeros, the gathers served by L2 (every problem). MFS_SWEEP_STAGED: one CTA per
   group of columns (rows), the gathered vector streamed through shared memory in 64 KB blocks and
   the nonzeros stored sorted by block (FP32_MIXED solvers; Lorentz cones of at most 64 columns are
   projected in the column pass's epilogue, larger ones by their own kernel as in the chunked
   sweeps). MFS_SWEEP_AUTO (default): where the staged layout is built on the GPU (COO input in
   column order) for a matrix with at least 2^20 nonzeros, the staged column pass if it has at
   least 8 nonzeros per row and the staged row pass if it has at least 4 per column; chunked
   otherwise. All compute the same iteration; their FP32 sums run in different orders. */
enum { MFS_SWEEP_AUTO = 0, MFS_SWEEP_CHUNKED = 1, MFS_SWEEP_STAGED = 2 };

typedef struct {
    int32_t kind;  /* MFS_CONE_NONNEG or MFS_CONE_SOC */
    int32_t pad_;  /* ignored */
    int64_t size;  /* >= 1; the sizes of all cones sum to n */
} mfs_cone;

typedef struct {
    double mu;            /* ADMM penalty, > 0 (the paper's fixed mu; default 1) */
    int32_t check_every;  /* mfs_solve evaluates residuals every this many iterations (default 25) */
    int32_t precision;    /* MFS_FP64 (default) or MFS_FP32_MIXED */
    int32_t polish_iters; /* FP32_MIXED: FP64 iterations run by mfs_solve once the FP32 sweep has
                             met the tolerance, or early if it stalls (default 50) */
    int32_t stop_rule;    /* MFS_STOP_KKT (default), MFS_STOP_SCS_L2 or MFS_STOP_OSQP_INF */
    double osqp_rel;      /* MFS_STOP_OSQP_INF: eps_rel / eps_abs, > 0 (default 10: the paper's
                             OSQP tolerances 1e-4 and 1e-3 at tol = 1e-4) */
    int32_t sweep;        /* MFS_SWEEP_AUTO (default; see above), MFS_SWEEP_CHUNKED, or
                             MFS_SWEEP_STAGED: build the staged layout (device memory of a second
                             copy of A) and use it for both passes; FP32_MIXED solvers only, FP64
                             ones run the chunked kernels (mfs_get_info tells) */
    int32_t adapt_mu;     /* 0 (default): mu stays fixed, the paper's method. k > 0: a variant outside
                             the paper (residual balancing): at the residual checks k, 2k, 4k, 8k, ...
                             of mfs_solve (exponentially spaced, so that mu changes finitely often),
                             mu doubles if max(r_prim, r_cone) > 5 r_dual and halves if
                             r_dual > 5 max(r_prim, r_cone), within [mu/256, 256 mu] of its value
                             when mfs_solve began (mfs_set_mu semantics: the iterate is kept).
                             Ignored by mfs_iterate and by the batch and shared-A solvers. */
    int32_t l2_keep;      /* 0 (default) or 1. The staged passes access the iterate's vectors with an L2
                             evict-last hint; such lines stay in L2 only within the context's persisting
                             set-aside (cudaLimitPersistingL2CacheSize). With 1 a solver that sets up
                             staged passes raises that limit to the device's maximum while it exists
                             (the last such solver to be destroyed puts the previous value back): the
                             large LP's iteration then takes 135 instead of 141 us, but all other work in
                             the CUDA context has that much less L2 meanwhile (the chunked sweeps of the
                             same instance: 184 instead of 118 us). Ignored by the batch and shared-A
                             solvers. */
} mfs_settings;

/* Residuals at the current (x, lambda); all accumulated in FP64.
   r_prim = ||Ax-b||_2/(1+||b||_2); r_cone = ||x-P_K x||_2/(1+||x||_2);
   r_dual = ||s-P_K s||_2/(1+||c||_2) with s = c + A^T lambda (K is self-dual, so this is the
   distance of the dual slack to the dual cone); r_gap = |c^T x + b^T lambda|/(1+|c^T x|+|b^T lambda|);
   kkt = max of the four.
   The paper's two other rules (Sec. V), read for a problem whose variable lies in a cone: the
   constraint x in K joins the equality rows, its distance ||x - P_K x|| joining the primal residual,
   and the dual residual c + A^T lambda is taken after subtracting its projection on K (the cone
   multiplier), so that both vanish at an optimum of an LP or SOCP.
   r_scs  = max( sqrt(||Ax-b||_2^2 + ||x-P_K x||_2^2)/(1+||b||_2), ||s-P_K s||_2/(1+||c||_2), r_gap );
   r_osqp = max( max(||Ax-b||_inf, ||x-P_K x||_inf) / (1 + q max(||Ax||_inf, ||x||_inf, ||b||_inf)),
                 ||s-P_K s||_inf / (1 + q max(||A^T lambda||_inf, ||c||_inf)) ),  q = settings.osqp_rel;
   so that r_osqp <= tol is the paper's OSQP test with eps_abs = tol, eps_rel = q tol.
   The raw norms follow (nrm_*: l2, inf_*: infinity norm). */
typedef struct {
    double r_prim, r_dual, r_cone, r_gap, kkt, pobj, dobj;
    double nrm_res_p, nrm_b, nrm_xdist, nrm_x, nrm_sdist, nrm_c, nrm_atl_c;
    double inf_res_p, inf_ax, inf_b, inf_atl_c, inf_atl, inf_c;
    double inf_x, inf_xdist, inf_sdist; /* ||x||_inf, ||x-P_K x||_inf, ||s-P_K s||_inf */
    double r_scs, r_osqp;
    int64_t iter; /* iterations run since mfs_create or the last mfs_warm_start */
} mfs_residuals_t;

typedef struct {
    int64_t m, n, o;            /* o = stored nonzeros after summing duplicates, dropping zeros */
    int64_t ncones, nsoc, nbig; /* cones; Lorentz cones; Lorentz cones too large to fuse */
    int64_t col_chunks, row_chunks;
    int64_t bytes_per_iter;     /* algorithmic HBM bytes of one iteration at the current precision */
    int32_t precision;          /* precision the iterate is currently held in */
    int32_t launches_per_iter;  /* kernel launches of one iteration (sweeps, long chunks, big cones) */
    int32_t sweep_col, sweep_row; /* MFS_SWEEP_CHUNKED or MFS_SWEEP_STAGED: kernels of the column and
                                     row passes at the current precision */
    int32_t col_parts, row_parts; /* staged passes: CTAs per column (row) group, each streaming its
                                     share of the gathered vector into partial sums that a combine
                                     kernel adds in a fixed order (1: no split); 0 without staged passes */
} mfs_info_t;

/* Defaults: mu = 1, check_every = 25, precision = MFS_FP64, polish_iters = 50, stop_rule =
   MFS_STOP_KKT, osqp_rel = 10, sweep = MFS_SWEEP_AUTO, adapt_mu = 0. */
void mfs_default_settings(mfs_settings* s);

/*
 * Build a solver (Algorithm 1, steps 1-3: the UV decomposition and the diagonal factors).
 * m, n >= 0; nnz >= 0 COO triplets in any order (host): row[t] in [0,m), col[t] in [0,n),
 * val[t] finite. Duplicates are summed and entries that are (or sum to) exactly zero are dropped.
 * b (m doubles, host), c (n doubles, host); cones: ncones entries whose sizes sum to n.
 * settings may be NULL (defaults). cuda_stream: a cudaStream_t or NULL. Limits: m, n, o < 2^31.
 * The iterate starts at zero (x = z = delta = lambda = 0, which is Algorithm 1 started from
 * y = gamma = 0). On success *out receives the handle; on failure *out is NULL.
 * Set-up: with 2^16 or more entries the COO list is copied to the device once and checked there.
 * Host threads narrow the indices to int32 on the way (each checked against its range first) and
 * copy through pinned staging buffers that the process keeps after the first such call (64 MB of
 * pinned host memory, one stream per copy thread; mfs_get_solution uses them too). If the list is
 * in column order (rows ascending within a column, duplicates next to each other) the orders and
 * padded layouts are built on the GPU, taking about 60 bytes of device memory per entry until the
 * call returns. Otherwise the host orders it with all its cores. The result is the same either way.
 */
mfs_status mfs_create(int64_t m, int64_t n, int64_t nnz, const int64_t* row, const int64_t* col,
                      const double* val, const double* b, const double* c, int64_t ncones,
                      const mfs_cone* cones, const mfs_settings* settings, void* cuda_stream,
                      mfs_solver** out);

/*
 * Same as mfs_create, for a problem whose data are already in device memory (for instance torch
 * tensors), so that they make no trip through the host: row, col (nnz int64 each), val (nnz
 * doubles), b (m doubles) and c (n doubles) are device pointers of the current device; cones and
 * settings stay host memory. The same rules and results as mfs_create: indices checked on the
 * device (MFS_ERR_INVALID naming the first entry out of range, or a non-finite value in A, b or c),
 * duplicates summed, zeros dropped. COO in column order (rows ascending within a column, duplicates
 * next to each other) is set up on the device alone; any other order is copied to the host once
 * and ordered there (the host path of mfs_create). The arrays are only read, and may be freed or
 * reused once the call has returned.
 */
mfs_status mfs_create_device(int64_t m, int64_t n, int64_t nnz, const int64_t* row, const int64_t* col,
                             const double* val, const double* b, const double* c, int64_t ncones,
                             const mfs_cone* cones, const mfs_settings* settings, void* cuda_stream,
                             mfs_solver** out);

/* Release all device and host memory of the handle. NULL is ignored. */
void mfs_destroy(mfs_solver* s);

/* One-line description of the last failure on this handle ("" if none). NULL gives the last
   failure of mfs_create on this thread. The string lives until the next call on the handle. */
const char* mfs_last_error(const mfs_solver* s);

mfs_status mfs_get_info(const mfs_solver* s, mfs_info_t* out);

/* Choose the sweep kernels of the FP32 iteration: MFS_SWEEP_AUTO, MFS_SWEEP_CHUNKED or
   MFS_SWEEP_STAGED (see above). MFS_ERR_INVALID for an unknown kind, or for MFS_SWEEP_STAGED on a
   solver whose staged layout was not built (neither requested by settings.sweep = MFS_SWEEP_STAGED
   nor chosen by MFS_SWEEP_AUTO, or in FP64). The iterate is kept; FP64 iterations always use the
   chunked kernels. */
mfs_status mfs_set_sweep(mfs_solver* s, int32_t kind);

/* Diagnostic of the bounded waits of the staged sweeps: runs one staged column pass that issues
   no copies and gives up after a few polls of each wait. Returns MFS_ERR_TIMEOUT when the kernel
   reported the give-up (the expected result) and clears the flag; the FP32 iterate is overwritten
   and must be reset (mfs_warm_start) before further use. MFS_ERR_INVALID without staged sweeps. */
mfs_status mfs_debug_staged_wait_test(mfs_solver* s);

/* Bounds-checked build (libmfs_bounds.so, compiled with MFS_DEBUG_BOUNDS): the single-instance sweep
   and residual kernels check every gather index, padded-entry load and shared-memory index, skip
   an access that fails (reading 0) and record the first failure. mfs_debug_bounds returns 1 in
   that build and 0 otherwise; *site (nullable) receives the failed check's site (0: none so far;
   1 padded entries, 2 v gathered by the column sweep, 3 x by the row sweep, 4 lambda by the
   column residual, 5 x by the row residual, 6/7/8 the staged vector block, segment sums and
   entries) and *index (nullable) the low 40 bits of the index; reset clears the record. */
int32_t mfs_debug_bounds(int64_t* site, int64_t* index, int32_t reset);

/* Change mu (Algorithm 1 takes mu fixed; F_U and F_V do not depend on it, so no set-up is
   repeated). The iterate is kept. mu must be > 0. */
mfs_status mfs_set_mu(mfs_solver* s, double mu);

/*
 * Warm start from a primal-dual point (Algorithm 1 accepts any initial point). Host arrays of
 * doubles: x (n) and lambda (m) are required; z (n) and delta (n) may be NULL, which selects
 * z = proj_K(x) and delta = proj_K(c + A^T lambda). The iterate becomes the state that
 * Algorithm 1 reaches after an iteration ending at (x, lambda): gamma = -U^T lambda and
 * y = V^T x + U^T F_U (b - A x). Resets the iteration counter.
 */
mfs_status mfs_warm_start(mfs_solver* s, const double* x, const double* lambda, const double* z,
                          const double* delta);

/* Same as mfs_warm_start, with device pointers to doubles. */
mfs_status mfs_warm_start_device(mfs_solver* s, const double* x, const double* lambda,
                                 const double* z, const double* delta);

/* Start from an arbitrary point of Algorithm 1 (its Require line: x, z, delta in R^n, y, gamma in
   R^o, lambda in R^m), all host FP64 arrays, required. y and gamma follow Algorithm 1's nonzero
   order k: columns in turn, rows ascending within each column, over the o nonzeros of the stored A
   (duplicates summed, explicit zeros dropped; o as in mfs_info_t). The next two iterations run the
   literal updates of Algorithm 1 on the o-length y and gamma; after them gamma = -U^T lambda and
   y = V^T x + U^T F_U (b - A x) hold, and the solver continues with its reduced sweeps, so every
   iterate equals Algorithm 1's from that start. Resets the iteration count. MFS_ERR_INVALID for a
   NULL array; changing the precision is refused until the two literal iterations have run. */
mfs_status mfs_warm_start_literal(mfs_solver* s, const double* x, const double* y, const double* z,
                                  const double* gamma, const double* delta, const double* lambda);

/* Run exactly k >= 0 iterations (Algorithm 1, steps 5-10) with no termination test. */
mfs_status mfs_iterate(mfs_solver* s, int64_t k);

/*
 * Iterate until the measure of the settings' stopping rule (mfs_residuals_t.kkt, .r_scs or
 * .r_osqp) is <= tol, testing every check_every iterations, or until max_iter more iterations
 * have run. Returns MFS_OK (tolerance
 * met) or MFS_MAX_ITER; MFS_ERR_NUMERIC if the residuals become NaN/Inf. iters_out (nullable)
 * receives the iterations run by this call. In FP32_MIXED mode the iterate switches to FP64
 * (and stays there) for the final polish_iters iterations, or as soon as the FP32 residual has
 * not improved over 40 consecutive checks; the tolerance is always tested on FP64 reductions.
 * Primal infeasibility: when Ax = b, x in K has no solution, lambda grows along a direction d
 * with A^T d in K* (= K) and b^T d < 0 (Farkas). At every check the change d of lambda since the
 * previous check is tested: dist(A^T d, K) <= 0.1 |b^T d|, b^T d < -1e-3 ||b|| ||d||, and the
 * primal residual not 1 % lower than three checks before; three consecutive passes return
 * MFS_INFEASIBLE (the iterate is kept). Unbounded primal: x then grows along a ray e with A e = 0,
 * e in K and c^T e < 0; with e the change of x since the previous check, ||A e|| <= 0.1 |c^T e|,
 * dist(e, K) <= 0.1 |c^T e|, c^T e < -1e-3 ||c|| ||e|| and a stalled dual residual, three
 * consecutive passes return MFS_UNBOUNDED.
 */
mfs_status mfs_solve(mfs_solver* s, double tol, int64_t max_iter, int64_t* iters_out);

/* One residual check of mfs_solve: iterations run by that call when it was made, the relative
   residuals (as in mfs_residuals_t), the stopping rule's measure, the precision of the iterate and
   the penalty mu from then on. */
typedef struct {
    int64_t iter;
    double kkt, r_prim, r_dual, r_cone, r_gap, measure;
    int32_t precision;
    int32_t reserved;
    double mu;  /* mu of the iterations that follow the check (after any residual-balancing change) */
} mfs_check_t;

/* The checks of the last mfs_solve on this handle (a ring of the most recent 4096): the latest
   min(capacity, kept) records, oldest first, into out; *count (nullable) receives the number of
   checks that call made. Host-only; no device work. */
mfs_status mfs_solve_history(const mfs_solver* s, mfs_check_t* out, int64_t capacity, int64_t* count);

/* Residuals of the current iterate (FP64 reductions on the device). */
mfs_status mfs_residuals(mfs_solver* s, mfs_residuals_t* out);

/* Copy the iterate to host arrays of doubles: x, z, delta (n each), lambda (m). Any may be NULL. */
mfs_status mfs_get_solution(mfs_solver* s, double* x, double* lambda, double* z, double* delta);

/* The fifth vector of the reduced state (see the top of this file), v = F_U (b - A x) - lambda/mu
   as the last row pass left it (m doubles, host): with (x, z, delta, lambda) it fixes every later
   iterate (Algorithm 1's y and gamma are y = V^T x + U^T (v + lambda/mu), gamma = -U^T lambda).
   MFS_ERR_INVALID while a literal start (mfs_warm_start_literal) has not yet run its two
   iterations. */
mfs_status mfs_get_reduced_v(mfs_solver* s, double* v);

/* Same as mfs_get_solution, into device arrays of doubles. */
mfs_status mfs_get_solution_device(mfs_solver* s, double* x, double* lambda, double* z,
                                   double* delta);

/* Switch the iterate between FP32 and FP64 storage (MFS_FP32_MIXED handles only; converting
   FP32 -> FP64 is exact, FP64 -> FP32 rounds to nearest). */
mfs_status mfs_set_precision(mfs_solver* s, int32_t precision);

/*
 * Measurement hook: run k iterations with each kernel launched on its own (no graph), back to
 * back, bracketed by CUDA events on the solver's stream, and wait once at the end. out_ms[0] = average milliseconds of one
 * column-order sweep kernel, out_ms[1] = of one row-order sweep kernel, out_ms[2] = of the
 * large-cone kernel (0 if none), out_ms[3] = average milliseconds of one whole iteration.
 * The iterate advances by k iterations.
 */
mfs_status mfs_time_kernels(mfs_solver* s, int64_t k, double* out_ms);

/* The same, kernel by kernel: out_ms[0..5] = average milliseconds of the column pass's main kernel
   (the staged kernel or the chunked sweep), of its second kernel (the combine of a pass in parts, or
   the long-column kernel; 0 if none), of the large-cone kernel, of the row pass's main kernel, of its
   second kernel (combine or long rows), and of a whole iteration. An event between two kernels ends
   their overlap (programmatic dependent launch), so the sum can exceed an iteration without them. */
mfs_status mfs_time_kernel_split(mfs_solver* s, int64_t k, double* out_ms);

/* ------------------------------------------------------------------------------------------------
 * Batched solves. Many independent problems (Sec. II form each, Algorithm 1 on each) of uneven
 * sizes are solved in one persistent launch: every CTA takes instances from a queue (largest
 * first) and iterates one instance at a time with the vectors that its sweeps gather from held in
 * shared memory (and the instance's matrix too when it fits). The launch is captured in a CUDA
 * graph and replayed.
 * ---------------------------------------------------------------------------------------------- */
typedef struct mfs_batch mfs_batch;

typedef struct {
    int32_t threads;      /* threads per CTA: 128, 256 or 512 */
    int32_t ctas_per_sm;  /* 1..4 resident CTAs per SM (each gets 1/ctas_per_sm of the shared memory) */
    int32_t check_every;  /* iterations between an instance's residual checks in mfs_batch_solve */
    int32_t reserved;
} mfs_batch_tuning;

/*
 * count >= 1 instances. Instance t has m[t] rows, n[t] columns, nnz[t] COO entries and ncones[t]
 * cones; all per-instance arrays are concatenated in instance order (host): row/col/val (sum of
 * nnz entries, indices local to the instance), b (sum of m), c (sum of n), cones (sum of ncones).
 * Entry and cone rules as for mfs_create. settings: mu, check_every and precision (FP64, or
 * FP32_MIXED = FP32 sweep with FP64 residual reductions) are used; polish_iters is ignored.
 * Iterates start at zero. Default tuning: 256 threads, 1 CTA per SM.
 */
mfs_status mfs_batch_create(int64_t count, const int64_t* m, const int64_t* n, const int64_t* nnz,
                            const int64_t* row, const int64_t* col, const double* val,
                            const double* b, const double* c, const int64_t* ncones,
                            const mfs_cone* cones, const mfs_settings* settings, void* cuda_stream,
                            mfs_batch** out);
void mfs_batch_destroy(mfs_batch* bt);
/* Like mfs_last_error, for batches; NULL gives the last mfs_batch_create failure on this thread. */
const char* mfs_batch_last_error(const mfs_batch* bt);
/* Bytes of each stored local index of A (2 when every instance has m, n <= 65535, else 4): a nonzero
   then costs 2 * (4 + bytes) in FP32 (both orders) instead of 16. */
mfs_status mfs_batch_index_bytes(const mfs_batch* bt, int32_t* bytes);
mfs_status mfs_batch_get_info(const mfs_batch* bt, int64_t* count, int64_t* total_m, int64_t* total_n,
                              int64_t* total_nnz);
/* Exactly k iterations of every instance (no termination test). */
mfs_status mfs_batch_iterate(mfs_batch* bt, int64_t k);
/* Each instance iterates until its relative KKT residual (as in mfs_residuals_t) is <= tol, checked
   every check_every iterations inside the launch, or until max_iter iterations. iters and status
   (nullable, count entries each) receive per instance the iterations run by this call and MFS_OK or
   MFS_MAX_ITER. */
mfs_status mfs_batch_solve(mfs_batch* bt, double tol, int64_t max_iter, int64_t* iters, int32_t* status);
/* FP64 residuals of every instance at its current iterate; out has count entries. */
mfs_status mfs_batch_residuals(mfs_batch* bt, mfs_residuals_t* out);
/* Iterate of instance t as doubles (host arrays; any may be NULL): x, z, delta (n[t]), lambda (m[t]). */
mfs_status mfs_batch_get_solution(mfs_batch* bt, int64_t t, double* x, double* lambda, double* z,
                                  double* delta);
mfs_status mfs_batch_set_tuning(mfs_batch* bt, const mfs_batch_tuning* tuning);
mfs_status mfs_batch_get_tuning(const mfs_batch* bt, mfs_batch_tuning* tuning);
/* Autotuner: times `iters` iterations of the whole batch for each candidate (threads per CTA x CTAs
   per SM) and keeps the fastest; then, with that launch shape, times max(iters, 400) iterations with
   the in-launch residual checks every 10, 25, 50, 100 or 200 iterations and keeps the smallest
   interval whose checks cost at most 5 % more than every 200 (a finer interval stops each instance
   closer to its first iteration at the tolerance). Returns the choice in chosen (nullable). The
   iterate advances. */
mfs_status mfs_batch_tune(mfs_batch* bt, int64_t iters, mfs_batch_tuning* chosen);

/* ------------------------------------------------------------------------------------------------
 * Ruiz equilibration of the data, a convergence variant outside the paper (Algorithm 1 runs on the
 * data as given): D. Ruiz's scaling (2001). Host functions; the caller creates a solver of any kind
 * on the scaled data and maps its solution back.
 * ---------------------------------------------------------------------------------------------- */
/* passes of: take the infinity norms of the rows and of the columns of the current matrix over the
   listed COO entries (the columns of one Lorentz cone share the largest of their norms, so that the
   cone is scaled as one block and stays a cone), then divide every row and column by the square root
   of its norm (a zero norm leaves it alone); each entry is multiplied by its row factor, then by its
   column factor. In place: val (nnz) becomes A' = D A E, b (m) becomes D b, c (n) becomes E c; d (m)
   and e (n) receive the diagonals of D and E. Same argument rules as mfs_create (indices in range,
   finite values, cones summing to n) -> MFS_ERR_INVALID with mfs_ruiz_last_error() set, before
   anything is written. Repeated (row, column) entries count separately in the norms. */
mfs_status mfs_ruiz_scale(int64_t m, int64_t n, int64_t nnz, const int64_t* row, const int64_t* col, double* val,
                          double* b, double* c, int64_t ncones, const mfs_cone* cones, int32_t passes, double* d,
                          double* e);
/* The original problem's point from the scaled problem's, in place (any of x, z, delta (n), lambda (m)
   may be NULL): x = E x', z = E z', lambda = D lambda', delta = E^-1 delta'. */
mfs_status mfs_ruiz_unscale(int64_t m, int64_t n, const double* d, const double* e, double* x, double* lambda,
                            double* z, double* delta);
/* The inverse map, for a start of the original problem given to a solver of the scaled one. */
mfs_status mfs_ruiz_scale_start(int64_t m, int64_t n, const double* d, const double* e, double* x, double* lambda,
                                double* z, double* delta);
const char* mfs_ruiz_last_error(void);

/* ------------------------------------------------------------------------------------------------
 * Shared-A solves: count problems with one constraint matrix A and cone K and their own b and c
 * (a parametric family), iterated together. The instances' vectors are interleaved so that each
 * nonzero's gather serves 32 instances with one coalesced load.
 * ---------------------------------------------------------------------------------------------- */
typedef struct mfs_shared mfs_shared;

/* A (COO, host, rules as mfs_create) and K once; count >= 1 instances; b and c start at zero
   until mfs_shared_set_data. settings: mu, check_every, precision are used. */
mfs_status mfs_shared_create(int64_t m, int64_t n, int64_t nnz, const int64_t* row, const int64_t* col,
                             const double* val, int64_t ncones, const mfs_cone* cones, int64_t count,
                             const mfs_settings* settings, void* cuda_stream, mfs_shared** out);
void mfs_shared_destroy(mfs_shared* sh);
const char* mfs_shared_last_error(const mfs_shared* sh);
/* b [count][m] and c [count][n]: host doubles, or device floats for the _device form. Also resets
   every iterate to zero. */
mfs_status mfs_shared_set_data(mfs_shared* sh, const double* b, const double* c);
mfs_status mfs_shared_set_data_device(mfs_shared* sh, const float* b, const float* c);
/* Zero start for every instance. */
mfs_status mfs_shared_reset(mfs_shared* sh);
/* Warm start of every instance from device floats x [count][n], lambda [count][m] (as
   mfs_warm_start with z and delta defaulted). */
mfs_status mfs_shared_warm_start_device(mfs_shared* sh, const float* x, const float* lambda);
mfs_status mfs_shared_iterate(mfs_shared* sh, int64_t k);
/* Residuals of every instance (out: count entries). */
mfs_status mfs_shared_residuals(mfs_shared* sh, mfs_residuals_t* out);
/* Iterate everything, testing each instance every check_every iterations, until all have relative
   KKT residual <= tol or max_iter iterations ran. iters (nullable, count entries): the iteration at
   which each instance first met tol, or -1. MFS_OK if all met it, else MFS_MAX_ITER. */
mfs_status mfs_shared_solve(mfs_shared* sh, double tol, int64_t max_iter, int64_t* iters);
/* Iterate, instance-major, device floats: x [count][n], lambda [count][m] (either may be NULL). */
mfs_status mfs_shared_get_solution_device(mfs_shared* sh, float* x, float* lambda);
/* Continuous batching: members enter and leave single slots while the other slots iterate on.
   slots: host array of count distinct slot numbers in [0, count of the handle). load_slots gives
   those slots new data, b [count][m] and c [count][n] as device FP32 rows in the order of slots,
   and the zero start (x = z = delta = lambda = 0); the other slots are untouched. get_slots_device
   copies those slots' x [count][n] and lambda [count][m] into device FP32 arrays (either may be
   NULL). Both synchronous; MFS_ERR_INVALID for a bad slot list. */
mfs_status mfs_shared_load_slots(mfs_shared* sh, int64_t count, const int32_t* slots, const float* b,
                                 const float* c);
mfs_status mfs_shared_get_slots_device(mfs_shared* sh, int64_t count, const int32_t* slots, float* x,
                                       float* lambda);
/* load_slots followed, for those slots only, by the warm start of mfs_shared_warm_start_device:
   x [count][n] and lambda [count][m] (device FP32 rows in the order of slots, required) become the
   iterate, z = proj_K(x), delta = proj_K(c + A^T lambda), v = F_U (b - A x) - lambda/mu. The other
   slots are untouched. Synchronous. */
mfs_status mfs_shared_load_slots_warm(mfs_shared* sh, int64_t count, const int32_t* slots, const float* b,
                                      const float* c, const float* x, const float* lambda);
/* Iterate of instance t as host doubles (any may be NULL): x, z, delta (n), lambda (m). */
mfs_status mfs_shared_get_solution(mfs_shared* sh, int64_t t, double* x, double* lambda, double* z,
                                   double* delta);

/* ------------------------------------------------------------------------------------------------
 * Learned warm start. The paper has no counterpart; this serves parametric families of problems:
 * a 3-layer MLP theta (din) -> width -> width -> dout (ReLU after the first two layers) maps a
 * problem's parameters to a starting point (for instance x and lambda concatenated, dout = n + m)
 * for mfs_warm_start. Weights are FP32 masters with BF16 copies; every GEMM runs on the tcgen05
 * tensor cores (BF16 inputs, FP32 accumulation); training minimises the mean squared error
 * against standardised targets with Adam. All x, y, target pointers are device FP32 arrays,
 * row-major [batch][features]. Calls are synchronous on the handle's stream.
 * ---------------------------------------------------------------------------------------------- */
typedef struct mfs_mlp mfs_mlp;

/* din, width, max_batch: positive multiples of 8, max_batch <= 65535; dout >= 1. Weights He-uniform
   from seed. */
mfs_status mfs_mlp_create(int32_t din, int32_t width, int32_t dout, int32_t max_batch, uint64_t seed,
                          void* cuda_stream, mfs_mlp** out);
void mfs_mlp_destroy(mfs_mlp* net);
const char* mfs_mlp_last_error(const mfs_mlp* net);
/* Targets are standardised per output as (t - mean) / std; host arrays of dout floats. */
mfs_status mfs_mlp_set_output_scaling(mfs_mlp* net, const float* mean, const float* stdv);
/* Sets the standardisation from a device target matrix [count][dout] (row-major FP32): per output,
   mean and standard deviation over the rows (FP64 sums), the deviation raised to min_std (> 0) where
   it is smaller, so that outputs constant over the data stay finite. Synchronous. */
mfs_status mfs_mlp_fit_output_scaling(mfs_mlp* net, int64_t count, const float* targets, float min_std);
/* Host copies of the current mean and std (dout floats each); NULL skips. */
mfs_status mfs_mlp_get_output_scaling(mfs_mlp* net, float* mean, float* stdv);
/* y = net(x) for batch <= max_batch rows; denormalize != 0 undoes the standardisation. */
mfs_status mfs_mlp_forward(mfs_mlp* net, int32_t batch, const float* x, float* y, int32_t denormalize);
/* Mean squared error of one batch (batch a multiple of 8) and its gradients, kept in the handle;
   loss (nullable, host) receives the loss. */
mfs_status mfs_mlp_backward(mfs_mlp* net, int32_t batch, const float* x, const float* target, double* loss);
/* Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the gradients of the last mfs_mlp_backward. */
mfs_status mfs_mlp_adam_step(mfs_mlp* net, float lr);
/* The update of mfs_mlp_backward followed by mfs_mlp_adam_step, with the output layer fused into
   the tensor-core GEMM epilogues: the forward GEMM of layer 3 produces the loss gradient instead of
   the output, and the weight-gradient GEMM of layer 3 applies Adam in place (so mfs_mlp_get_grads
   does not report layer 3's weights after this call unless mfs_mlp_keep_grads is on). */
mfs_status mfs_mlp_train_step(mfs_mlp* net, int32_t batch, const float* x, const float* target, float lr,
                              double* loss);
/* Host copies of layer l (0..2): weights [out][in] and bias; NULL skips. */
mfs_status mfs_mlp_get_params(mfs_mlp* net, int32_t layer, float* W, float* b);
mfs_status mfs_mlp_set_params(mfs_mlp* net, int32_t layer, const float* W, const float* b);
mfs_status mfs_mlp_get_grads(mfs_mlp* net, int32_t layer, float* gW, float* gb);
/* Adam state of layer l (0..2), host copies: first (mW) and second (vW) moments of the weights
   [out][in], of the bias (mb, vb); any may be NULL. *step (nullable) receives the number of Adam
   steps taken, the t of the bias corrections 1 - beta^t of the next step minus one. */
mfs_status mfs_mlp_get_adam_state(mfs_mlp* net, int32_t layer, float* mW, float* vW, float* mb, float* vb,
                                  int64_t* step);
/* The BF16 copy of layer l's weights [out][in] that the tensor-core GEMMs read, as raw 16-bit
   patterns (host array of out*in). */
mfs_status mfs_mlp_get_weights_bf16(mfs_mlp* net, int32_t layer, uint16_t* Wh);
/* on != 0: mfs_mlp_train_step also stores the weight gradient of layer 3 that its fused Adam
   epilogue consumes, so that mfs_mlp_get_grads reports it (one more FP32 store per weight). */
mfs_status mfs_mlp_keep_grads(mfs_mlp* net, int32_t on);

/* Dense GEMM on the tensor cores: C[M x N] = A[M x K] * B[N x K]^T (+ bias[N], then ReLU if relu),
   A and B row-major BF16 device arrays (K a multiple of 8), C row-major FP32 (out_fp32) or BF16,
   bias nullable FP32. splits > 1 splits K over that many CTAs per tile (deterministic sum).
   Synchronous; allocates its split workspace on the stream. */
mfs_status mfs_gemm_bf16(int64_t M, int64_t N, int64_t K, const void* A, const void* B, const float* bias,
                         int32_t relu, int32_t out_fp32, void* C, int32_t splits, void* cuda_stream);

/* Fault injection for tests: after n more successful device allocations (by any handle of this
   library in the process), every further one fails as if the device were out of memory, so each
   create call's failure path (MFS_ERR_OOM, everything allocated so far freed) can be exercised.
   n < 0 disarms it. Not thread-safe with respect to the allocations it counts. */
mfs_status mfs_debug_fail_alloc_after(int64_t n);

/* Diagnostic of the bounded waits: runs the tensor-core GEMM on a 128 x 128 x 64 problem with its
   loads switched off and a short poll limit, so that the MMA issuer's first wait runs out, first in
   the one-tile kernel, then in the persistent kernel of the fused epilogues (the loss epilogue,
   whose epilogue warps' waits run out as well). Each kernel records the time-out and returns
   normally (no trap, no hang; its tensor memory is freed); the call returns MFS_ERR_TIMEOUT when
   both do, and the context stays usable.
   Allocates and frees its own small buffers; synchronous on cuda_stream (NULL = legacy stream). */
mfs_status mfs_gemm_bf16_wait_test(void* cuda_stream);

/*
 * mfs_row_residuals_static -- row-side residuals of a point (x, lambda) without allocating.
 * The paper has no counterpart: this is a service for callers that cannot allocate device memory
 * when they need a residual (a framework that owns all device memory through its own pool and
 * forbids side allocations, plugin hosts whose execute callbacks must not allocate, real-time
 * loops that allocate only at start-up). It needs no solver handle and calls no cudaMalloc,
 * cudaFree or other allocating routine.
 *
 * All pointers are device pointers of the current device. A is given in CSR form: row_ptr
 * (m+1 int32 offsets), col_idx and val (row_ptr[m] entries; col_idx in [0,n)); b and lambda hold
 * m doubles, x holds n doubles. out receives 8 doubles:
 *   {r_prim, ||Ax-b||_2, ||Ax-b||_inf, ||Ax||_inf, ||b||_2, ||b||_inf, b^T lambda, -b^T lambda}
 * (the same quantities as the matching fields of mfs_residuals_t), FP64, deterministic.
 *
 * Unlike the calls above it is asynchronous: the work is enqueued on cuda_stream (NULL = legacy
 * default stream) and the call returns without waiting; read out after synchronizing.
 * Scratch: a static 1 MiB device array that every GPU which loads this library holds until the
 * process exits. Limit: m <= 4,194,304 rows; a larger m returns MFS_ERR_INVALID and enqueues
 * nothing, as do negative sizes, n >= 2^31 - 1 and a NULL array among out, row_ptr, col_idx, val, b
 * and lambda (m > 0) or x (n > 0). Set-up: the array's device address belongs to the current
 * context and is looked up (cudaGetSymbolAddress) by every call whose stream is not being
 * captured; while a capture is under way the address found by the last call in the same context
 * is reused (MFS_ERR_INVALID if there was none), so the first call in each context should come
 * before any stream capture.
 * Every call uses the same array: calls whose work can overlap on the GPU (different streams,
 * or different host threads) race on it, so the caller must order them. No state carries over
 * between calls (each call writes every scratch slot it reads). If an error from earlier work is
 * already pending on the calling thread (cudaPeekAtLastError), the call returns MFS_ERR_CUDA,
 * enqueues nothing and leaves that error in place; MFS_ERR_CUDA also if the device lookup or one
 * of its own launches fails.
 */
mfs_status mfs_row_residuals_static(int64_t m, int64_t n, const int32_t* row_ptr, const int32_t* col_idx,
                                    const double* val, const double* b, const double* x,
                                    const double* lambda, double* out, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* MFS_H */
