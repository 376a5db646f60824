/*
 * gpcg_oracle.h -- interface of the FP64 CPU oracle for GPCG.
 *
 * TEST INFRASTRUCTURE ONLY: used by the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark; never by the CUDA library.
 */
#ifndef GPCG_ORACLE_H
#define GPCG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Status codes (numbering independent of the CUDA library's). */
enum {
    ORA_OK = 0,
    ORA_ERR_NUMERIC = 3,    /* <p, A p> <= 0 or a non-finite value */
    ORA_ERR_MAXIT = 7,      /* max_outer reached before the tau test held */
    ORA_ERR_LINESEARCH = 8  /* max_ls halvings without sufficient decrease */
};

/* Why a gradient projection phase ended. */
enum { ORA_GP_SAME_FACE = 1 /* pgstop1 */, ORA_GP_PROGRESS = 2 /* pgstop2 */, ORA_GP_MAXIT = 3 };

/* Why a conjugate gradient phase ended. */
enum { ORA_CG_EMPTY = 0, ORA_CG_PROGRESS = 1 /* cgstop1 */, ORA_CG_EXACT = 2, ORA_CG_MAXIT = 3 };

/* Trace event kinds. */
enum {
    ORA_EV_START = 1,   /* a = q(x0), b = ||pg(x0)||, c = tau */
    ORA_EV_GP_STEP = 2, /* inner = j, trials, a = alpha, b = q(y_{j-1}) - q(y_j), c = same face, d = ||pg|| */
    ORA_EV_GP_END = 3,  /* inner = j, a = reason, b = alpha0 of the last step */
    ORA_EV_CG_ITER = 4, /* inner = j, a = alpha, b = Delta_j, c = <r_j, z_j>, d = <p, A p> */
    ORA_EV_CG_END = 5,  /* inner = iterations, a = reason, b = eta2 in force */
    ORA_EV_SEARCH = 6,  /* trials, a = alpha, b = q(x_{k+1}) - q(x_k), c = ||pg||, d = (B == A) */
    ORA_EV_DONE = 7     /* outer = iterations, a = status, b = ||pg||, c = q */
};

typedef struct {
    int dim;              /* 2 or 3 */
    int64_t nx, ny, nz;   /* nz = 1 when dim == 2; point i = ix + nx*(iy + ny*iz) */
    const double* diag;   /* A(i,i) */
    const double* cx;     /* A(i,i+1) */
    const double* cy;     /* A(i,i+nx) */
    const double* cz;     /* A(i,i+nx*ny), dim == 3 only */
} ora_stencil;

/* Preconditioners of the reduced CG (Sec. 6 compares them).  TILE: block
 * Jacobi with one block per 64 x 8 tile of each xy-plane (tiles start at
 * multiples of 64 in x and 8 in y; couplings between tiles and between planes
 * are dropped), each block solved approximately by one symmetric zebra line
 * Gauss-Seidel sweep: exact solves along the x-lines of the tile's even rows,
 * then its odd rows, then its even rows again, each line with the current
 * values of its neighbouring lines on the right-hand side.  That is
 * M = (D + L) D^-1 (D + U) per tile, D the line tridiagonals, L/U the
 * couplings between lines in the order (even rows, odd rows). */
enum {
    ORA_PRECOND_NONE = 0,
    ORA_PRECOND_JACOBI = 1, /* M = diag(A_k) */
    ORA_PRECOND_TILE = 2    /* tile block Jacobi, zebra line sweep */
};
enum { ORA_TILE_X = 64, ORA_TILE_Y = 8 };

typedef struct {
    double tau_abs, tau_rel;
    double eta1, eta2, mu, eta2_shrink, eta2_floor;
    int max_outer, max_gp, max_cg, max_ls;
    int precond;          /* ORA_PRECOND_* */
} ora_options;

typedef struct {
    double q, pg_norm, pg_norm0;
    int64_t n_active, n_binding, n_free;
    int outer_iters, gp_iters, cg_iters, ls_trials;
    int status;
} ora_stats;

typedef struct {
    int64_t n_active, n_binding;
    double pg_norm2, q;
} ora_census_out;

typedef struct {
    int kind, outer, inner, trials;
    double a, b, c, d;
} ora_event;

/* Threads for the loops whose rows are independent (results do not depend on
 * the count; reductions always run on one thread).  t <= 0: all processors.
 * Without OpenMP the count stays 1. */
void ora_set_threads(int t);
int ora_get_threads(void);

void ora_default_options(ora_options* o);
void ora_matvec(const ora_stencil* A, const double* x, double* y);
void ora_masked_matvec(const ora_stencil* A, const uint8_t* free_mask, const double* p,
                       double* y);
double ora_q(const ora_stencil* A, const double* b, double c, const double* x);
void ora_project(int64_t n, const double* l, const double* u, const double* x, double* out);
void ora_proj_gradient(int64_t n, const double* x, const double* g, const double* l,
                       const double* u, double* pg);
void ora_census(const ora_stencil* A, const double* b, double c, const double* l,
                const double* u, const double* x, double* g, uint8_t* active,
                ora_census_out* out);
int ora_gp_step(const ora_stencil* A, const double* b, const double* l, const double* u,
                double mu, int max_ls, double* y, double* g, double* alpha0,
                double* alpha, double* decrease, int* trials);
int ora_reduced_cg(const ora_stencil* A, const uint8_t* free_mask, const double* g,
                   double eta2, int max_cg, int precond, double* w, int* iters, int* reason,
                   ora_event* events, int64_t event_cap, int64_t* event_len);
/* z = M^-1 r on the free set (zero elsewhere) for preconditioner `precond`. */
void ora_precondition(const ora_stencil* A, const uint8_t* free_mask, int precond,
                      const double* r, double* z);
int ora_projected_search(const ora_stencil* A, const double* b, const double* l,
                         const double* u, double mu, int max_ls, const double* d,
                         double* x, double* g, double* alpha, double* dq, int* trials);
int ora_gpcg(const ora_stencil* A, const double* b, double c, const double* l,
             const double* u, const double* x0, const ora_options* opt, double* x,
             ora_stats* st, ora_event* events, int64_t event_cap, int64_t* event_len);

#ifdef __cplusplus
}
#endif
#endif
