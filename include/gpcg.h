/*
 * gpcg.h -- C ABI of the GB300 GPCG library (libgpcg.so).
 *
 * GPCG solves the bound-constrained strictly convex quadratic program
 *
 *     min { q(x) = 1/2 x'Ax + b'x + c  :  l <= x <= u }
 *
 * (Benson, McInnes & More, "GPCG: a case study in the performance and
 * scalability of optimization algorithms", Sec. 2, Eq. def_bqp, def_bounds,
 * def-quadratic) by alternating gradient projection with conjugate gradients
 * on the face of the current iterate (Sec. 3, Algorithm GPCG).  A is a
 * symmetric positive definite 2-D 5-point or 3-D 7-point stencil.  Every
 * numerical step runs in the library's own CUDA kernels on the current
 * device; the library never falls back to the CPU.
 *
 * Conventions for every entry point:
 *   - Pointers to arrays may be host or device pointers (the library asks the
 *     CUDA runtime which); arrays are dense, contiguous, FP64, indexed
 *     i = ix + nx*(iy + ny*iz) with ix fastest.  Input arrays are only read,
 *     and only during the call; the library keeps its own device copies.
 *   - Every call returns a gpcg_status; nothing is thrown across the ABI.
 *     gpcg_last_error() gives a one-line description of the latest failure
 *     on the calling thread.
 *   - Handles are owned by the library and released only by the matching
 *     _destroy call.  A handle must not be used from two threads at once;
 *     distinct handles may be used concurrently.
 *   - Infinite bounds are written as -INFINITY / +INFINITY.
 *   - The padded point count px*ny*nz, with px = nx rounded up to a multiple
 *     of 8, must be below 2^31 (so n = nx*ny*nz is too); larger problems are
 *     refused with GPCG_ERR_ARG before any array is read.
 */
#ifndef GPCG_H
#define GPCG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GPCG_OK = 0,
    GPCG_ERR_ARG = 1,         /* invalid argument (NULL, bad size, NaN, diag <= 0, ...) */
    GPCG_ERR_INFEASIBLE = 2,  /* some l_i > u_i, l_i = +inf or u_i = -inf: Omega is empty */
    GPCG_ERR_NUMERIC = 3,     /* a curvature <p,Ap> <= 0 (A not SPD) or a non-finite value */
    GPCG_ERR_OOM = 4,         /* device allocation failed */
    GPCG_ERR_BUDGET = 5,      /* request larger than the server's HBM budget */
    GPCG_ERR_CUDA = 6,        /* a CUDA runtime call failed */
    GPCG_ERR_MAXIT = 7,       /* max_outer iterates without ||grad_Omega q|| <= tau */
    GPCG_ERR_LINESEARCH = 8,  /* max_ls halvings without sufficient decrease */
    GPCG_ERR_TIMEOUT = 9,     /* the host-side pass cap was reached */
    GPCG_ERR_PENDING = 10,    /* result not available yet (solve not run / still running) */
    GPCG_ERR_CANCELLED = 11   /* request cancelled before it finished */
} gpcg_status;

/* Precision modes.
 *   GPCG_FP64: every vector, coefficient and reduction in FP64.
 *   GPCG_MIXED: two phases.
 *     1. An FP32 phase runs Algorithm GPCG on an FP32 copy of the iterate,
 *        kept inside the FP32 box [RN(l), RN(u)]: coefficients, vectors,
 *        gradient, projection and search directions are FP32, and a point
 *        is active when its FP32 value equals its FP32 bound bit for bit.
 *        Each thread sums its FP32 products over a chunk of rows in FP32 and
 *        folds the chunk sums into compensated (float-float) accumulators,
 *        which are reduced over the grid and converted to FP64; the CG step
 *        lengths, the
 *        Armijo comparisons (Eq. gplsstop, cglsstop2), q(x) and the phase's
 *        tau test are FP64 decisions on those sums.  The phase ends at its
 *        first tau hit, after a failed projected search, or when ||pg||
 *        stops decreasing (FP32 noise).
 *     2. An FP64 phase: an FP64 census rebuilds x (the FP64 bound where the
 *        FP32 value sat at its FP32 bound, else the FP64 projection) and
 *        recomputes g, the active and binding sets, q and ||pg|| in FP64;
 *        with refine, one CG phase on that face (eta2 reduced) and an FP64
 *        projected search follow; GPCG then continues in FP64 until the FP64
 *        tau test holds.  The CG phases of the FP64 phase run in FP64
 *        (refine 1) or, as correction solves on the FP64 gradient, in FP32
 *        streams with the same compensated sums (refine 2).  The returned x, its statistics and the final
 *        termination test are FP64.
 *   gpcg_stats.mixed_n_active and fp64_gp_iters tell whether the FP64 phase
 *   changed the face the FP32 phase identified. */
typedef enum {
    GPCG_FP64 = 0,
    GPCG_MIXED = 1
} gpcg_precision;

/* The Hessian as stencil bands (Sec. 2: A symmetric positive definite).
 * diag[i] = A(i,i); cx[i] = A(i,i+1); cy[i] = A(i,i+nx); cz[i] = A(i,i+nx*ny)
 * (dim == 3 only).  The entry of the last point along an axis (ix = nx-1 for
 * cx, ...) is ignored.  Each array holds n values. */
typedef struct {
    int dim;               /* 2 or 3 */
    int64_t nx, ny, nz;    /* grid size; nz must be 1 when dim == 2 */
    const double* diag;
    const double* cx;
    const double* cy;
    const double* cz;      /* NULL when dim == 2 */
} gpcg_stencil;

typedef struct gpcg_problem gpcg_problem;

/* Create a problem (Sec. 4: the TaoSetQuadraticFunction / TaoSetVariableBounds
 * pair).  Copies A, b, l, u to library-owned device memory and checks them:
 * sizes, no NaN, finite couplings, diag > 0, l <= u, l < +inf, u > -inf.
 * l == NULL means l = -inf everywhere, u == NULL means u = +inf everywhere.
 * On success *out receives the handle; on failure *out is set to NULL.
 * Errors: GPCG_ERR_ARG, GPCG_ERR_INFEASIBLE, GPCG_ERR_OOM, GPCG_ERR_CUDA. */
gpcg_status gpcg_problem_create(const gpcg_stencil* A, const double* b, const double* l,
                                const double* u, double c, gpcg_problem** out);

/* Replace the data of a problem by a QP of the same grid (A->dim, nx, ny, nz
 * equal to the problem's): the bands, b, l, u and c, with the same meaning,
 * checks and error statuses as gpcg_problem_create (on an error the
 * problem's data are undefined, and solves report GPCG_ERR_ARG, until the
 * next successful update).  The
 * problem keeps its device memory, tensor maps and launch graphs, so a
 * stream of QPs of one shape pays for the copies of its data and nothing
 * else.  gpcg_result reports GPCG_ERR_PENDING until the next solve. */
gpcg_status gpcg_problem_update(gpcg_problem* p, const gpcg_stencil* A, const double* b,
                                const double* l, const double* u, double c);

/* gpcg_problem_update without waiting: the copies are enqueued on `stream`
 * (a cudaStream_t; page-locked host arrays make them asynchronous) and the
 * call returns.  The arrays must stay valid until those copies are done.
 * The device-side set-up and the value checks run on the stream of the next
 * call that uses the problem's data (a solve, a masked product, ...).  That
 * call waits for the checks before it computes anything; a failed check
 * makes it return GPCG_ERR_ARG or GPCG_ERR_INFEASIBLE, and every later call
 * on the problem does the same until the next update.  With two problems
 * used in turn, the next QP's copies overlap the current solve.
 * Errors at the call: GPCG_ERR_ARG, GPCG_ERR_CUDA. */
gpcg_status gpcg_problem_update_async(gpcg_problem* p, const gpcg_stencil* A, const double* b,
                                      const double* l, const double* u, double c,
                                      void* stream);

/* Release every resource of the handle (NULL is allowed). */
void gpcg_problem_destroy(gpcg_problem* p);

/* Problem size n = nx*ny*nz (0 for NULL). */
int64_t gpcg_problem_size(const gpcg_problem* p);

/* Solver options.  Defaults come from gpcg_default_options():
 * tau_abs 0, tau_rel 1e-8 (stop when ||grad_Omega q(x)|| <= max(tau_abs,
 * tau_rel*||grad_Omega q(x0)||), Eq. bqp_approximate_sol, 2-norm);
 * eta1 0.1 (Eq. pgstop2), eta2 0.05 (Eq. cgstop1) -- the values of Sec. 5;
 * mu 0.01 (Eq. gplsstop / cglsstop2, the paper only asks mu in (0,1/2));
 * eta2_shrink 0.1 and eta2_floor 1e-12 (the reduction of eta2 when Eq.
 * cgstop3 holds, unspecified in the paper); max_outer 10000, max_gp 50,
 * max_cg 10000, max_ls 60; precision GPCG_FP64; refine 2; x0 NULL (start at
 * P[l], falling back to u then 0 where a bound is infinite: Sec. 5 uses
 * x0 = l); cuda_stream NULL (the legacy default stream); lambda_min 0;
 * precond GPCG_PRECOND_NONE; cg_system GPCG_CG_MASKED; path
 * GPCG_PATH_AUTO. */
typedef struct {
    double tau_abs, tau_rel;
    double eta1, eta2, mu, eta2_shrink, eta2_floor;
    int max_outer, max_gp, max_cg, max_ls;
    int precision;          /* gpcg_precision */
    int refine;             /* GPCG_MIXED, after the FP32 phase: 0 no closing CG phase;
                               1 the closing CG phase and every later one in FP64;
                               2 every later CG phase in FP32 streams on the FP64
                               gradient (a correction solve: mixed-precision iterative
                               refinement, the FP64 search and census deciding) */
    const double* x0;       /* optional start (host or device, n values), projected onto Omega */
    void* cuda_stream;      /* cudaStream_t the solve is ordered on */
    double lambda_min;      /* optional lower bound on lambda_min(A), for err_bound */
    int precond;            /* gpcg_precond: preconditioner of the CG phase (Sec. 6) */
    int cg_system;          /* gpcg_cg_system: how the CG phase applies A_k (Sec. 4) */
    int path;               /* gpcg_path: which solver runs the problem */
} gpcg_options;

/* Which solver runs a problem of gpcg_solve / gpcg_solve_batch.
 *   GPCG_PATH_AUTO (default): the resident solver when the problem fits it,
 *     else the pass engine.
 *   GPCG_PATH_ENGINE: the pass engine (persistent passes over the grid, one
 *     launch per pass), whatever the size.
 *   GPCG_PATH_RESIDENT: the resident solver; GPCG_ERR_ARG when the problem
 *     does not fit it.
 * The resident solver runs the whole of Algorithm GPCG for one problem in
 * one thread block, every vector in shared memory: problems of at most 2048
 * points whose FP64 arrays (and, in GPCG_MIXED, their FP32 copies) fit one
 * block's 227 KB of shared memory (about 1200 points in mixed precision,
 * 1800 in FP64), with GPCG_PRECOND_NONE or GPCG_PRECOND_JACOBI and
 * GPCG_CG_MASKED.  It follows the same algorithm, readings and precision
 * modes as the engine; its sums reduce in another fixed order, so its path
 * can differ from the engine's where a test is marginal.  In a batch every
 * fitting problem gets its own block in one launch, next to the engine's
 * run of the others; each result is still the same as solving that problem
 * alone with the same options.  The server always uses the engine. */
typedef enum {
    GPCG_PATH_AUTO = 0,
    GPCG_PATH_ENGINE = 1,
    GPCG_PATH_RESIDENT = 2
} gpcg_path;

/* How the CG phase works on the reduced system A_k = Z_k' A Z_k (Sec. 4).
 *   GPCG_CG_MASKED (default): full-length vectors, the free set a bitmask
 *     applied inside the stencil product (the paper's alternative technique).
 *   GPCG_CG_EXTRACTED: A_k is extracted, as the paper's design does: the free
 *     points get a compact numbering (tiles in order, rows within a tile,
 *     columns within a row), A_k is stored as rows of a diagonal and 2*dim
 *     neighbour slots in that numbering, and CG runs on compact vectors; w is
 *     scattered back before the projected search.  Three extra passes per CG
 *     phase; pays when few points are free.  Not with GPCG_PRECOND_TILE
 *     (GPCG_ERR_ARG).  The first solve with it allocates the compact arrays
 *     (capacity n: 4 + 4 dim bytes per point plus (9 + 2 dim) values per
 *     point of each CG precision). */
typedef enum { GPCG_CG_MASKED = 0, GPCG_CG_EXTRACTED = 1 } gpcg_cg_system;

/* Preconditioners of the CG phase on the reduced system (Sec. 6 compares the
 * diagonal one with block Jacobi); the decrease of Eq. cgstop1 is then
 * alpha_j <r_j, M^-1 r_j> / 2.
 *   GPCG_PRECOND_JACOBI: M = diag(A_k), the diagonal of the reduced Hessian.
 *   GPCG_PRECOND_TILE: block Jacobi with one block per 64 x 8 tile of the grid
 *     (tiles start at multiples of 64 in x and 8 in y; couplings between tiles
 *     are dropped), the analogue of the paper's one block per processor; each
 *     block is solved approximately by one symmetric zebra line Gauss-Seidel
 *     sweep on the free set (exact solves along the x-lines of the tile's even
 *     rows, then odd rows, then even rows), so M = (D + L) D^-1 (D + U) per
 *     tile, which is symmetric positive definite.  M^-1 is applied in FP32
 *     arithmetic in every precision mode.  2-D problems only, on the staged
 *     path (not with GPCG_NO_TMA); otherwise gpcg_solve returns GPCG_ERR_ARG.
 *     The first solve with it allocates 4 more vectors of the CG precision(s)
 *     (z = M^-1 r and q = M^-1 Ap, double-buffered). */
typedef enum {
    GPCG_PRECOND_NONE = 0,
    GPCG_PRECOND_JACOBI = 1,
    GPCG_PRECOND_TILE = 2
} gpcg_precond;

void gpcg_default_options(gpcg_options* o);

/* Run GPCG (Sec. 3, Algorithm GPCG) on one problem; blocks until it ends.
 * Returns the solve's status (GPCG_OK when the tolerance was met).
 * On the pass engine every pass of the solve runs in one cooperative kernel
 * launch (all blocks resident; a grid barrier between passes), except with
 * GPCG_CG_EXTRACTED, when the launch is refused, or when the environment
 * sets GPCG_NO_COOP=1: the passes then run as launches of a CUDA graph, with
 * bit-identical results.  Solves may be issued from several host threads on
 * their own streams; the cooperative kernels of one device run one at a
 * time. */
gpcg_status gpcg_solve(gpcg_problem* p, const gpcg_options* opt);

/* Run GPCG on `count` independent problems at once: every pass of the engine
 * advances all of them in one kernel launch (per-instance tile table).  The
 * result of each problem is bit-identical to solving it alone with the same
 * options.  Returns GPCG_OK if every solve met its tolerance, else the first
 * failing status; per-problem statuses are in gpcg_result(). */
gpcg_status gpcg_solve_batch(gpcg_problem* const* probs, int count, const gpcg_options* opt);

typedef struct {
    double q;               /* q(x) */
    double pg_norm;         /* ||grad_Omega q(x)||_2 (Eq. proj-gradient) */
    double pg_norm0;        /* ||grad_Omega q(x0)||_2 */
    double tau;             /* the tolerance in force */
    int64_t n_active, n_binding, n_free;   /* |A(x)|, |B(x)|, n - |A(x)| (Sec. 2) */
    int outer_iters, gp_iters, cg_iters, ls_trials;
    int refine_cg_iters;    /* CG iterations of the closing FP64 phase (GPCG_MIXED) */
    int passes;             /* engine passes (one HBM sweep each) */
    int status;             /* gpcg_status of the solve */
    double err_bound;       /* ||x - x*|| <= pg_norm / lambda_min when lambda_min > 0, else -1 */
    double alg_bytes;       /* algorithmic HBM bytes of all passes of the solve (the bytes
                               each pass must read and write once, summed) */
    int64_t launches;       /* kernel launches of the engine for the latest solve: 1 when
                               all its passes ran in one cooperative launch (a solve with
                               one engine instance, the default), else the passes plus the
                               empty launches of the final loop iteration; for a batch,
                               the launches of the whole batch */
    int staged;             /* the shared-memory (TMA) staged paths available to the problem:
                               1 free-set words, 2 FP64 CG passes, 4 FP32 CG passes,
                               8 mixed-precision gradient-projection passes (2-D only; the
                               other passes and 3-D problems use the register sweep) */
    int fp64_gp_iters;      /* GPCG_MIXED: gradient projection steps taken in FP64 after
                               the FP32 phase (0 in FP64 mode) */
    int64_t mixed_n_active; /* GPCG_MIXED: |A(x)| at the first FP64 census after the FP32
                               phase, i.e. the face that phase identified (-1 in FP64
                               mode).  The closing CG phase and projected search only add
                               points to the active set (the step is zero on it), so
                               mixed_n_active == n_active with fp64_gp_iters == 0 means
                               the FP32 phase found the returned face exactly. */
    int path;               /* the solver that ran: GPCG_PATH_ENGINE or GPCG_PATH_RESIDENT
                               (whose passes count 1: one launch, one read of the
                               problem and one write of the result) */
    int reserved;
} gpcg_stats;

/* Copy the latest solution (n values, host or device x_out; NULL skips it)
 * and statistics (NULL skips them): q(x) (Eq. def-quadratic), the projected
 * gradient norm ||grad_Omega q(x)|| (Eq. proj-gradient) the termination test
 * of Eq. bqp_approximate_sol compares with tau, and the sizes of the active
 * set A(x) and binding set B(x) (Sec. 2), all evaluated in FP64 at the
 * returned x; the iteration counts of Algorithm GPCG (Sec. 3).
 * GPCG_ERR_PENDING before the first solve. */
gpcg_status gpcg_result(const gpcg_problem* p, double* x_out, gpcg_stats* stats);

/* y = Z Z' A Z Z' p on the free set given by free_mask (one byte per point,
 * nonzero = free): the reduced Hessian A_k = Z_k' A Z_k of Eq. cg2 applied in
 * place, without extracting A_k (the "alternative technique" of Sec. 4).  This
 * runs the same kernel as the CG phase's matrix-vector product.  precision
 * GPCG_MIXED streams FP32 coefficients and vectors (p is rounded to FP32,
 * y is FP32 widened to FP64).  *pAp (optional) receives <p_F, (A_k p)_F>
 * accumulated in FP64.  Arrays: n values each, host or device. */
gpcg_status gpcg_masked_spmv(gpcg_problem* p, const uint8_t* free_mask, const double* pv,
                             double* y, double* pAp, int precision, void* cuda_stream);

/* The explicit reduced system of GPCG_CG_EXTRACTED for the free set given by
 * free_mask (one byte per point, nonzero = free), built by the same passes
 * as in a solve: *m receives the number of free points; fidx (m values) the
 * point (row-major index ix + nx*(iy + ny*iz)) of each compact index; diag
 * (m values) the diagonal; nb and val (2*dim*m values, slot-major: slot j of
 * compact row k at j*m + k; slots x-1, x+1, y-1, y+1, z-1, z+1) the
 * neighbours' compact indices and couplings, a slot outside the free set
 * holding the row's own index and 0.  Host arrays of capacity n (fidx,
 * diag) and 2*dim*n (nb, val).  precision GPCG_MIXED returns the FP32
 * rows widened to FP64.  Overwrites the problem's CG vectors (gpcg_result
 * reports GPCG_ERR_PENDING until the next solve). */
gpcg_status gpcg_reduced_system(gpcg_problem* p, const uint8_t* free_mask, int precision,
                                int64_t* m, int32_t* fidx, double* diag, int32_t* nb,
                                double* val, void* cuda_stream);

/* z = M^-1 r for the tile preconditioner (GPCG_PRECOND_TILE) on the free set
 * given by free_mask (one byte per point, nonzero = free): the pass that
 * starts a tile-preconditioned CG phase, run once on r in place of the
 * gradient.  z is 0 off the free set.  precision GPCG_MIXED rounds r to FP32
 * and returns FP32 values widened to FP64 (M^-1 itself is applied in FP32 in
 * both modes).  *rz (optional) receives <r_F, z_F> accumulated in FP64.
 * Arrays: n values each, host or device.  2-D problems on the staged path
 * only (GPCG_ERR_ARG otherwise).  Overwrites the problem's CG vectors, so
 * gpcg_result reports GPCG_ERR_PENDING until the next solve. */
gpcg_status gpcg_tile_precondition(gpcg_problem* p, const uint8_t* free_mask, const double* r,
                                   double* z, double* rz, int precision, void* cuda_stream);

/* Time `reps` launches of the masked matrix-vector kernel (the CG pass that
 * forms p and A_k p) on the problem's free set after the latest solve (or all
 * points free before any solve), with CUDA events on the given stream.  With
 * flush_l2 != 0 every launch is preceded by a write of 256 MiB (twice the L2
 * cache) so that each launch streams its operands from HBM, and only the
 * launches are timed.  *ms_per_launch receives the mean launch duration and
 * *bytes_per_launch the algorithmic bytes moved per launch (bands, r and p
 * read once, p and A_k p written once, the mask bits). */
gpcg_status gpcg_time_masked_spmv(gpcg_problem* p, int precision, int reps, int flush_l2,
                                  void* cuda_stream, double* ms_per_launch,
                                  double* bytes_per_launch);

/* Throughput of the masked matrix-vector kernel of Eq. cg2 (y = Z Z' A Z Z' p
 * and <p_F, y_F>) in a stream of launches, as an iterative method issues
 * them: `count` distinct problems (2 <= count <= 64, 2-D, on the staged
 * path) are multiplied in turn, `reps` rounds, back to back on the given
 * stream.  Each launch takes one CTA per SM and waits for the previous one
 * (another problem's) only before its final sum, so up to three consecutive
 * products stream at the same time: launch latency, the first copies and the
 * final reduction's tail overlap the stream's other work instead of adding to
 * each launch.  With distinct problems whose
 * operands together exceed the L2 cache, every launch streams its operands
 * from HBM.  The operand of each problem is that of gpcg_time_masked_spmv
 * (the latest solve's free set and p, else all points free and p = 1); one
 * untimed launch per problem precedes the timed region, which one event pair
 * brackets.  *ms_per_launch receives the timed region over reps * count and
 * *bytes_per_launch the mean algorithmic bytes of a launch (as for
 * gpcg_time_masked_spmv).  Errors: GPCG_ERR_ARG (NULL, count out of range, a
 * problem given twice, a 3-D problem or one off the staged path),
 * GPCG_ERR_TIMEOUT (a bounded wait gave up), GPCG_ERR_CUDA. */
gpcg_status gpcg_time_masked_spmv_stream(gpcg_problem** probs, int count, int precision,
                                         int reps, void* cuda_stream, double* ms_per_launch,
                                         double* bytes_per_launch);

/* The product of gpcg_masked_spmv (FP64) for callers that cannot allocate
 * device memory: processes whose device memory belongs entirely to their own
 * pool allocator, and latency-critical loops that cannot take the device-wide
 * synchronisation that cudaMalloc / cudaFree may cause.  The paper has no
 * counterpart; this is a deployment variant of the reduced-Hessian product.
 *
 * Computes y = Z Z' A Z Z' p and, if pAp != NULL, writes <p_F, y_F> to the
 * host or device address pAp (the call then waits for the stream, so pAp
 * must be NULL while the stream is being captured: GPCG_ERR_ARG otherwise).
 * A's bands, free_mask (one byte per point, nonzero = free), p and y must be
 * device pointers owned by the caller; y must not overlap any of the inputs
 * (GPCG_ERR_ARG: other threads still read p where y is written).  Nothing is
 * copied or allocated.  The
 * only scratch is a fixed array of about 33 KB in device memory, held by every
 * GPU that loads the library until the process exits; it allows at most 4096
 * tiles of 64x32 points (for example 8.4e6 points on a 2-D grid), and larger
 * problems are rejected with GPCG_ERR_ARG.  The first call on a device looks
 * up that array's device address, so make the first call on each device
 * before any stream capture.  All calls on a device share the array: calls
 * whose kernels overlap on the GPU (different streams, other host threads)
 * race and must be serialised by the caller.
 * Errors: GPCG_ERR_ARG (NULL, host pointer, bad size, too large, y overlapping
 * an input, pAp during a capture), GPCG_ERR_CUDA. */
gpcg_status gpcg_masked_spmv_noalloc(const gpcg_stencil* A, const uint8_t* free_mask,
                                     const double* p, double* y, double* pAp,
                                     void* cuda_stream);

/* ---- continuous-batching server --------------------------------------- */

typedef struct gpcg_server gpcg_server;

/* A server owns one engine whose passes advance every admitted solve in one
 * kernel launch.  Requests are admitted when their device footprint fits in
 * hbm_budget bytes; at most max_live run at once, and as many more may have
 * their uploads in flight.  Finished solves are retired and their memory
 * released while others keep running.  Four worker threads of the server,
 * each on its own stream, copy requests in and results out while the passes
 * run; device memory comes from the server's stream-ordered pool.
 * Errors: GPCG_ERR_ARG, GPCG_ERR_OOM, GPCG_ERR_CUDA. */
gpcg_status gpcg_server_create(size_t hbm_budget, int max_live, const gpcg_options* opt,
                               gpcg_server** out);

/* Queue one request.  The arrays (host pointers) must stay valid until the
 * request completes; x_out (host, n values) receives the solution.  Page-
 * locked arrays are copied by DMA directly, pageable ones through the
 * workers' pinned staging buffers.  The values are checked on the device
 * when the request takes its slot: a NaN, a non-positive diagonal or an
 * empty box ends the request with GPCG_ERR_ARG or GPCG_ERR_INFEASIBLE (see
 * gpcg_server_stats).  *ticket identifies the request.  Errors: GPCG_ERR_ARG,
 * GPCG_ERR_BUDGET (the request alone exceeds the budget).
 * A server handle is the exception to the one-thread rule: submit, done,
 * stats, cancel, counts and timing may be called from any thread while one
 * thread steps it. */
gpcg_status gpcg_server_submit(gpcg_server* s, const gpcg_stencil* A, const double* b,
                               const double* l, const double* u, double c, double* x_out,
                               int64_t* ticket);

/* Advance the server: move finished requests out of and uploaded ones into
 * the engine's slots, run `passes` engine passes over the running slots,
 * admit what fits the budget (its upload starts on a worker) and hand what
 * finished to a worker for the read-back of x.  Returns after the passes
 * (submissions from other threads are not blocked meanwhile).  One thread at
 * a time steps a server: a concurrent call returns GPCG_ERR_ARG. */
gpcg_status gpcg_server_step(gpcg_server* s, int passes);

/* 1 if the ticket finished (its x_out and stats are final), else 0. */
int gpcg_server_done(gpcg_server* s, int64_t ticket);

/* Statistics of a finished ticket, plus its latency (submit to retirement,
 * seconds).  GPCG_ERR_PENDING while it runs. */
gpcg_status gpcg_server_stats(gpcg_server* s, int64_t ticket, gpcg_stats* st,
                              double* latency_s);

/* Cancel a request that has not finished.  Its x_out is not written, unless
 * a worker was already copying its result out. */
gpcg_status gpcg_server_cancel(gpcg_server* s, int64_t ticket);

/* Where a server's steps spent their time so far, cumulative seconds:
 * out[0] moving finished requests out of and uploaded ones into slots,
 * out[1] launching the passes, out[2] reading back results, out[3] starting
 * uploads (host side), out[4] waiting for the passes, out[5] device time of
 * the passes (CUDA events); out[6] steps, out[7] steps that ran passes.
 * out must hold 8 values.  Errors: GPCG_ERR_ARG. */
gpcg_status gpcg_server_timing(gpcg_server* s, double* out);

/* Counts of queued, running and finished requests. */
void gpcg_server_counts(gpcg_server* s, int* queued, int* running, int* finished);

void gpcg_server_destroy(gpcg_server* s);

/* One-line description of the latest error on the calling thread. */
const char* gpcg_last_error(void);

/* Library version string. */
const char* gpcg_version(void);

#ifdef __cplusplus
}
#endif
#endif
