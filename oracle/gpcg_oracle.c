/*
 * gpcg_oracle.c -- plain, slow, sequential FP64 reference implementation of
 * GPCG (gradient projection + conjugate gradient) for the bound-constrained
 * quadratic program
 *
 *     min { q(x) = 1/2 x'Ax + b'x + c  :  l <= x <= u }            (Sec. 2)
 *
 * with A a symmetric positive definite 2-D 5-point or 3-D 7-point stencil.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the oracle that the CUDA path is
 * checked against.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or
 * helper with the CUDA library and must never be linked into it.
 *
 * Every function follows one passage of Benson, McInnes & More, "GPCG: a case
 * study in the performance and scalability of optimization algorithms"
 * (2000), cited by section and equation label.  Every sum runs sequentially
 * in index order, and the file is compiled with -ffp-contract=off so that
 * every multiply and add is a separately rounded IEEE operation on every host.
 * Loops whose rows are independent (y = Ax, projections, vector updates) may
 * be split over OpenMP threads (ora_set_threads): each row is computed by the
 * same operations whichever thread runs it, so results are bit-identical for
 * every thread count.  Reductions (dot products, the census) are never split.
 *
 * Readings where the paper is silent (all documented in the design notes):
 *   - mu (Armijo constant, "some mu in (0,1/2)") defaults to 0.01.
 *   - the empty max in (pgstop2) / (cgstop1) at j = 1 means the test is not
 *     applied at the first step.
 *   - "reduce eta2 and continue with the conjugate gradient method"
 *     (cgstop3) means: the next outer iterate skips the gradient projection
 *     phase and restarts CG (w0 = 0) on the free set of x_{k+1}, with
 *     eta2 <- max(eta2 * eta2_shrink, eta2_floor); eta2 returns to its
 *     initial value whenever B(x_{k+1}) != A(x_{k+1}).
 *   - the termination test ||grad_Omega q|| <= tau (bqp_approximate_sol) is
 *     applied at x0, after every accepted gradient projection step and after
 *     every projected search; tau = max(tau_abs, tau_rel*||grad_Omega q(x0)||)
 *     in the Euclidean norm.
 *   - sufficient decrease is evaluated through the exact quadratic identity
 *     q(y+s) - q(y) = 1/2 <s, grad q(y) + grad q(y+s)>, which avoids the
 *     cancellation of forming q(y+s) and q(y) separately.
 *   - x_i == l_i, x_i == u_i are exact FP64 comparisons: the projection mid()
 *     returns l_i or u_i bit for bit, so the active set is exact.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "gpcg_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

/* Row loops run in parallel only above this many rows (below it a thread team
 * costs more than it saves). */
#define ORA_PAR_MIN 32768
#ifdef _OPENMP
#define ORA_ROWS _Pragma("omp parallel for schedule(static) if (n >= ORA_PAR_MIN)")
#else
#define ORA_ROWS
#endif

static int ora_threads = 1;

void ora_set_threads(int t)
{
#ifdef _OPENMP
    ora_threads = t > 0 ? t : omp_get_num_procs();
    omp_set_num_threads(ora_threads);
#else
    (void)t;
    ora_threads = 1;
#endif
}

int ora_get_threads(void) { return ora_threads; }

/* ------------------------------------------------------------------------ */
/* The Hessian A as a stencil.                                               */
/* cx[i] = A(i, i+1), cy[i] = A(i, i+nx), cz[i] = A(i, i+nx*ny); the entry of */
/* the last point along an axis is ignored.  A is symmetric, so the coupling */
/* to the west/south/below neighbour j is read as cx[j], cy[j], cz[j].       */
/* ------------------------------------------------------------------------ */

static int64_t ora_n(const ora_stencil* A) { return A->nx * A->ny * A->nz; }

/* Row i of y = A x, written out term by term (Sec. 2, A in def-quadratic). */
static double row_times(const ora_stencil* A, int64_t i, const double* x)
{
    const int64_t nx = A->nx, ny = A->ny, nz = A->nz;
    const int64_t ix = i % nx;
    const int64_t iy = (i / nx) % ny;
    const int64_t iz = i / (nx * ny);
    double s = A->diag[i] * x[i];
    if (ix > 0)      s += A->cx[i - 1] * x[i - 1];
    if (ix < nx - 1) s += A->cx[i] * x[i + 1];
    if (iy > 0)      s += A->cy[i - nx] * x[i - nx];
    if (iy < ny - 1) s += A->cy[i] * x[i + nx];
    if (A->dim == 3) {
        const int64_t sz = nx * ny;
        if (iz > 0)      s += A->cz[i - sz] * x[i - sz];
        if (iz < nz - 1) s += A->cz[i] * x[i + sz];
    }
    return s;
}

/* y = A x. */
void ora_matvec(const ora_stencil* A, const double* x, double* y)
{
    const int64_t n = ora_n(A);
    ORA_ROWS
    for (int64_t i = 0; i < n; i++) y[i] = row_times(A, i, x);
}

/* y = Z Z' A Z Z' p: the reduced Hessian A_k = Z'AZ of (cg2) applied to the
 * free components of p, scattered back to full length (free[i] != 0 marks a
 * free variable; rows and columns of active variables are dropped). */
void ora_masked_matvec(const ora_stencil* A, const uint8_t* free_mask,
                       const double* p, double* y)
{
    const int64_t n = ora_n(A);
    double* pz = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    ORA_ROWS
    for (int64_t i = 0; i < n; i++) pz[i] = free_mask[i] ? p[i] : 0.0;
    ORA_ROWS
    for (int64_t i = 0; i < n; i++) y[i] = free_mask[i] ? row_times(A, i, pz) : 0.0;
    free(pz);
}

static double dot(int64_t n, const double* a, const double* b)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s += a[i] * b[i];
    return s;
}

/* q(x) = 1/2 x'Ax + b'x + c  (def-quadratic). */
double ora_q(const ora_stencil* A, const double* b, double c, const double* x)
{
    const int64_t n = ora_n(A);
    double* Ax = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    ora_matvec(A, x, Ax);
    double s = 0.5 * dot(n, x, Ax) + dot(n, b, x) + c;
    free(Ax);
    return s;
}

/* Median of {l, u, x} for l <= u: the projection P[x] = mid(l, u, x) (Sec. 3). */
static double mid(double l, double u, double x)
{
    if (x < l) return l;
    if (x > u) return u;
    return x;
}

void ora_project(int64_t n, const double* l, const double* u, const double* x,
                 double* out)
{
    ORA_ROWS
    for (int64_t i = 0; i < n; i++) out[i] = mid(l[i], u[i], x[i]);
}

/* Projected gradient (proj-gradient).  A variable with l_i == u_i is fixed,
 * so its component is 0 (both sign cases of the definition apply). */
static double pg_component(double x, double g, double l, double u)
{
    const int at_l = (x == l), at_u = (x == u);
    if (at_l && at_u) return 0.0;
    if (at_l) return g < 0.0 ? g : 0.0;
    if (at_u) return g > 0.0 ? g : 0.0;
    return g;
}

void ora_proj_gradient(int64_t n, const double* x, const double* g,
                       const double* l, const double* u, double* pg)
{
    ORA_ROWS
    for (int64_t i = 0; i < n; i++) pg[i] = pg_component(x[i], g[i], l[i], u[i]);
}

/* Active set A(x) and binding set B(x) (Sec. 2). */
static int is_active(double x, double l, double u) { return x == l || x == u; }

static int is_binding(double x, double g, double l, double u)
{
    return (x == l && g >= 0.0) || (x == u && g <= 0.0);
}

/* Everything the algorithm needs to know about a point x in Omega:
 * g = Ax + b, the active flags, |A(x)|, |B(x)|, ||grad_Omega q(x)||^2 and
 * q(x).  Returns through *out. */
static void classify(int64_t n, const double* b, double c, const double* l,
                     const double* u, const double* x, const double* g,
                     uint8_t* active, ora_census_out* out)
{
    int64_t na = 0, nb = 0;
    double pg2 = 0.0, xg = 0.0, bx = 0.0;
    for (int64_t i = 0; i < n; i++) {
        active[i] = (uint8_t)is_active(x[i], l[i], u[i]);
        na += active[i];
        nb += is_binding(x[i], g[i], l[i], u[i]);
        const double p = pg_component(x[i], g[i], l[i], u[i]);
        pg2 += p * p;
        /* q = 1/2 <x, Ax> + <b, x> + c with Ax = g - b */
        xg += x[i] * (g[i] - b[i]);
        bx += b[i] * x[i];
    }
    out->n_active = na;
    out->n_binding = nb;
    out->pg_norm2 = pg2;
    out->q = 0.5 * xg + bx + c;
}

void ora_census(const ora_stencil* A, const double* b, double c, const double* l,
                const double* u, const double* x, double* g, uint8_t* active,
                ora_census_out* out)
{
    const int64_t n = ora_n(A);
    ora_matvec(A, x, g);
    ORA_ROWS
    for (int64_t i = 0; i < n; i++) g[i] = g[i] + b[i];
    classify(n, b, c, l, u, x, g, active, out);
}

/* ------------------------------------------------------------------------ */
/* Work space and trace                                                      */
/* ------------------------------------------------------------------------ */

typedef struct {
    ora_event* ev;
    int64_t cap;
    int64_t len;
} trace_t;

static void emit(trace_t* t, int kind, int outer, int inner, int trials, double a,
                 double b, double c, double d)
{
    if (t->ev && t->len < t->cap) {
        ora_event* e = &t->ev[t->len];
        e->kind = kind;
        e->outer = outer;
        e->inner = inner;
        e->trials = trials;
        e->a = a;
        e->b = b;
        e->c = c;
        e->d = d;
    }
    t->len++;
}

/* ------------------------------------------------------------------------ */
/* Sufficient-decrease trial shared by the gradient projection step (next-y, */
/* gplsstop) and the projected search (cglsstop2): the trial point is        */
/* xt = P[x + alpha*dir]; it is accepted when                                */
/*     q(xt) <= q(x) + mu <grad q(x), xt - x>.                               */
/* q(xt) - q(x) is formed as 1/2 <s, g + gt>, s = xt - x, gt = A xt + b,     */
/* which equals the difference exactly for a quadratic.                      */
/* Returns 1 if accepted; fills xt, gt, and *dq = q(xt) - q(x).              */
/* ------------------------------------------------------------------------ */
static int armijo_trial(const ora_stencil* A, const double* b, const double* l,
                        const double* u, const double* x, const double* g,
                        const double* dir, double alpha, double mu, double* xt,
                        double* gt, double* dq)
{
    const int64_t n = ora_n(A);
    ORA_ROWS
    for (int64_t i = 0; i < n; i++) xt[i] = mid(l[i], u[i], x[i] + alpha * dir[i]);
    ora_matvec(A, xt, gt);
    ORA_ROWS
    for (int64_t i = 0; i < n; i++) gt[i] = gt[i] + b[i];
    double gs = 0.0, sgg = 0.0;
    for (int64_t i = 0; i < n; i++) {
        const double s = xt[i] - x[i];
        gs += g[i] * s;
        sgg += s * (g[i] + gt[i]);
    }
    *dq = 0.5 * sgg;
    return *dq <= mu * gs;
}

/* One gradient projection iterate y_{j+1} = P[y_j - alpha_j grad q(y_j)]
 * (next-y) with alpha_j the first of alpha0 * (1/2)^i, i = 0, 1, ...,
 * satisfying (gplsstop), alpha0 the exact minimiser of the quadratic
 * alpha -> q(y - alpha grad_Omega q(y)) (bqpls):
 *     alpha0 = <pg, pg> / <pg, A pg>.
 * On entry y, g = grad q(y).  On exit (status ORA_OK) y and g hold the
 * accepted point and its gradient; *decrease = q(y_j) - q(y_{j+1}),
 * *alpha = accepted step, *trials = number of trial points evaluated. */
int ora_gp_step(const ora_stencil* A, const double* b, const double* l,
                const double* u, double mu, int max_ls, double* y, double* g,
                double* alpha0_out, double* alpha_out, double* decrease,
                int* trials)
{
    const int64_t n = ora_n(A);
    const size_t bytes = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double* pg = (double*)malloc(bytes);
    double* Apg = (double*)malloc(bytes);
    double* dir = (double*)malloc(bytes);
    double* yt = (double*)malloc(bytes);
    double* gt = (double*)malloc(bytes);
    int status = ORA_ERR_LINESEARCH;
    *trials = 0;

    ora_proj_gradient(n, y, g, l, u, pg);
    ora_matvec(A, pg, Apg);
    const double gg = dot(n, pg, pg);
    const double gAg = dot(n, pg, Apg);
    if (!(gAg > 0.0) || !isfinite(gg)) {
        status = ORA_ERR_NUMERIC;
        goto done;
    }
    const double alpha0 = gg / gAg;
    *alpha0_out = alpha0;
    ORA_ROWS
    for (int64_t i = 0; i < n; i++) dir[i] = -g[i];
    for (int i = 0; i <= max_ls; i++) {
        const double alpha = ldexp(alpha0, -i);
        double dq;
        (*trials)++;
        if (armijo_trial(A, b, l, u, y, g, dir, alpha, mu, yt, gt, &dq)) {
            memcpy(y, yt, bytes);
            memcpy(g, gt, bytes);
            *alpha_out = alpha;
            *decrease = -dq;
            status = ORA_OK;
            break;
        }
    }
done:
    free(pg);
    free(Apg);
    free(dir);
    free(yt);
    free(gt);
    return status;
}

/* Conjugate gradient on the reduced system (cg2):
 *     min q_k(w) = 1/2 <w, A_k w> + <r_k, w>,  A_k = Z'AZ, r_k = Z' g,
 * from w0 = 0, written in full-length vectors that are zero on the active
 * set.  Iteration j (1-based):
 *     alpha_j = ||r||^2 / <p, A_k p>,  w += alpha_j p,  r += alpha_j A_k p,
 *     Delta_j = q_k(w_{j-1}) - q_k(w_j) = 1/2 alpha_j ||r_{j-1}||^2,
 * the closed form of the decrease along a CG step (r_{j-1} orthogonal to
 * p_{j-2} so <r_{j-1}, p_{j-1}> = -||r_{j-1}||^2).  Stops at the first j >= 2
 * with Delta_j <= eta2 * max_{l<j} Delta_l (cgstop1), when r vanishes, or at
 * max_cg; the step of the stopping iteration is kept, so w = w_{j_k}.
 * Returns ORA_OK or ORA_ERR_NUMERIC (<p, A_k p> <= 0). */
/* Solve the tridiagonal system of the reduced Hessian along one x-line
 * segment: points i0 .. i0+len-1 of one row, couplings A(i,i+1) = cx[i]
 * between consecutive points that are both free, nothing outside the
 * segment.  A point off the free set gets the equation z_i = 0.  Thomas
 * algorithm (forward elimination, back substitution); cp and dp are scratch
 * of length len. */
static void line_solve(const ora_stencil* A, const uint8_t* fm, int64_t i0, int64_t len,
                       const double* rhs, double* z, double* cp, double* dp)
{
    for (int64_t k = 0; k < len; k++) {
        const int64_t i = i0 + k;
        const double a = (k > 0 && fm[i] && fm[i - 1]) ? A->cx[i - 1] : 0.0;
        const double c = (k + 1 < len && fm[i] && fm[i + 1]) ? A->cx[i] : 0.0;
        const double b = fm[i] ? A->diag[i] : 1.0;
        const double d = fm[i] ? rhs[k] : 0.0;
        const double den = k > 0 ? b - a * cp[k - 1] : b;
        cp[k] = c / den;
        dp[k] = k > 0 ? (d - a * dp[k - 1]) / den : d / den;
    }
    for (int64_t k = len - 1; k >= 0; k--) {
        z[i0 + k] = k + 1 < len ? dp[k] - cp[k] * z[i0 + k + 1] : dp[k];
    }
}

/* The tile preconditioner (ORA_PRECOND_TILE): in every 64 x 8 tile of every
 * xy-plane, z starts at 0 and the lines of the even rows, then the odd rows,
 * then the even rows are solved exactly with the couplings A(i, i +- nx) to
 * the rows above and below inside the tile moved to the right-hand side with
 * the current z there. */
static void tile_sweep(const ora_stencil* A, const uint8_t* fm, const double* r, double* z)
{
    const int64_t nx = A->nx, ny = A->ny, nz = A->nz;
    double* rhs = (double*)malloc(sizeof(double) * ORA_TILE_X);
    double* cp = (double*)malloc(sizeof(double) * ORA_TILE_X);
    double* dp = (double*)malloc(sizeof(double) * ORA_TILE_X);
    for (int64_t i = 0; i < nx * ny * nz; i++) z[i] = 0.0;
    for (int64_t iz = 0; iz < nz; iz++) {
        for (int64_t y0 = 0; y0 < ny; y0 += ORA_TILE_Y) {
            const int64_t y1 = y0 + ORA_TILE_Y < ny ? y0 + ORA_TILE_Y : ny;
            for (int64_t x0 = 0; x0 < nx; x0 += ORA_TILE_X) {
                const int64_t len = x0 + ORA_TILE_X < nx ? ORA_TILE_X : nx - x0;
                static const int parity[3] = {0, 1, 0};
                for (int h = 0; h < 3; h++) {
                    for (int64_t iy = y0 + parity[h]; iy < y1; iy += 2) {
                        const int64_t i0 = x0 + nx * (iy + ny * iz);
                        for (int64_t k = 0; k < len; k++) {
                            const int64_t i = i0 + k;
                            double v = r[i];
                            if (iy > y0 && fm[i] && fm[i - nx]) v -= A->cy[i - nx] * z[i - nx];
                            if (iy + 1 < y1 && fm[i] && fm[i + nx]) v -= A->cy[i] * z[i + nx];
                            rhs[k] = v;
                        }
                        line_solve(A, fm, i0, len, rhs, z, cp, dp);
                    }
                }
            }
        }
    }
    free(rhs);
    free(cp);
    free(dp);
}

/* z = M^{-1} r on the free set: the identity, the diagonal of the reduced
 * Hessian A_k (point Jacobi, Sec. 6), or the tile block Jacobi above (the
 * analogue of the paper's block Jacobi with one block per processor). */
static void precondition(const ora_stencil* A, const uint8_t* free_mask, int precond,
                         const double* r, double* z)
{
    const int64_t n = ora_n(A);
    if (precond == ORA_PRECOND_TILE) {
        tile_sweep(A, free_mask, r, z);
        return;
    }
    ORA_ROWS
    for (int64_t i = 0; i < n; i++) {
        if (!free_mask[i]) z[i] = 0.0;
        else if (precond == ORA_PRECOND_JACOBI) z[i] = r[i] / A->diag[i];
        else z[i] = r[i];
    }
}

void ora_precondition(const ora_stencil* A, const uint8_t* free_mask, int precond,
                      const double* r, double* z)
{
    precondition(A, free_mask, precond, r, z);
}

/* Preconditioned conjugate gradients on subproblem (cg2) from w_0 = 0, in
 * the textbook recurrences with rho_j = <r_j, z_j>, z_j = M^{-1} r_j:
 * alpha_j = rho_j / <p_j, A_k p_j>, w += alpha p, r += alpha A_k p,
 * beta = rho_{j+1} / rho_j, p = -z + beta p.  The decrease of q_k in step j
 * is alpha_j rho_j - alpha_j^2 <p_j, A_k p_j> / 2 = alpha_j rho_j / 2, which
 * feeds the test (cgstop1).  With M = I this is plain CG. */
static int reduced_cg(const ora_stencil* A, const uint8_t* free_mask, const double* g,
                      double eta2, int max_cg, int precond, double* w, int* iters,
                      int* reason, trace_t* tr, int outer)
{
    const int64_t n = ora_n(A);
    const size_t bytes = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double* r = (double*)malloc(bytes);
    double* z = (double*)malloc(bytes);
    double* p = (double*)malloc(bytes);
    double* Ap = (double*)malloc(bytes);
    int status = ORA_OK;
    ORA_ROWS
    for (int64_t i = 0; i < n; i++) {
        r[i] = free_mask[i] ? g[i] : 0.0;
        w[i] = 0.0;
    }
    precondition(A, free_mask, precond, r, z);
    ORA_ROWS
    for (int64_t i = 0; i < n; i++) p[i] = -z[i];
    double rr = dot(n, r, z);
    double dmax = 0.0;
    *iters = 0;
    *reason = ORA_CG_EMPTY;
    for (int j = 1; rr > 0.0 && j <= max_cg; j++) {
        ora_masked_matvec(A, free_mask, p, Ap);
        const double pAp = dot(n, p, Ap);
        if (!(pAp > 0.0)) {
            status = ORA_ERR_NUMERIC;
            break;
        }
        const double alpha = rr / pAp;
        ORA_ROWS
        for (int64_t i = 0; i < n; i++) {
            w[i] += alpha * p[i];
            r[i] += alpha * Ap[i];
        }
        const double delta = 0.5 * alpha * rr;
        precondition(A, free_mask, precond, r, z);
        const double rr_new = dot(n, r, z);
        *iters = j;
        if (tr) emit(tr, ORA_EV_CG_ITER, outer, j, 0, alpha, delta, rr_new, pAp);
        if (j >= 2 && delta <= eta2 * dmax) {
            *reason = ORA_CG_PROGRESS;
            break;
        }
        if (rr_new == 0.0) {
            *reason = ORA_CG_EXACT;
            break;
        }
        if (j == max_cg) {
            *reason = ORA_CG_MAXIT;
            break;
        }
        if (delta > dmax) dmax = delta;
        const double beta = rr_new / rr;
        ORA_ROWS
        for (int64_t i = 0; i < n; i++) p[i] = -z[i] + beta * p[i];
        rr = rr_new;
    }
    free(r);
    free(z);
    free(p);
    free(Ap);
    return status;
}

int ora_reduced_cg(const ora_stencil* A, const uint8_t* free_mask, const double* g,
                   double eta2, int max_cg, int precond, double* w, int* iters, int* reason,
                   ora_event* events, int64_t event_cap, int64_t* event_len)
{
    trace_t tr = {events, event_cap, 0};
    const int s = reduced_cg(A, free_mask, g, eta2, max_cg, precond, w, iters, reason, &tr, 0);
    if (event_len) *event_len = tr.len;
    return s;
}

/* Projected search along d (cglsstop2): x_{k+1} = P[x + alpha d] with alpha
 * the first of 1, 1/2, 1/4, ... satisfying sufficient decrease.  On exit x, g
 * hold the accepted point and gradient. */
int ora_projected_search(const ora_stencil* A, const double* b, const double* l,
                         const double* u, double mu, int max_ls, const double* d,
                         double* x, double* g, double* alpha_out, double* dq_out,
                         int* trials)
{
    const int64_t n = ora_n(A);
    const size_t bytes = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double* xt = (double*)malloc(bytes);
    double* gt = (double*)malloc(bytes);
    int status = ORA_ERR_LINESEARCH;
    *trials = 0;
    for (int i = 0; i <= max_ls; i++) {
        const double alpha = ldexp(1.0, -i);
        double dq;
        (*trials)++;
        if (armijo_trial(A, b, l, u, x, g, d, alpha, mu, xt, gt, &dq)) {
            memcpy(x, xt, bytes);
            memcpy(g, gt, bytes);
            *alpha_out = alpha;
            *dq_out = dq;
            status = ORA_OK;
            break;
        }
    }
    free(xt);
    free(gt);
    return status;
}

void ora_default_options(ora_options* o)
{
    o->tau_abs = 0.0;
    o->tau_rel = 1e-8;
    o->eta1 = 0.1;   /* Sec. 5: eta1 = 0.1 in (pgstop2) */
    o->eta2 = 0.05;  /* Sec. 5: eta2 = 0.05 in (cgstop1) */
    o->mu = 0.01;
    o->eta2_shrink = 0.1;
    o->eta2_floor = 1e-12;
    o->max_outer = 10000;
    o->max_gp = 50;
    o->max_cg = 10000;
    o->max_ls = 60;
    o->precond = ORA_PRECOND_NONE;
}

/* Algorithm GPCG (Sec. 3): gradient projection until (pgstop1) or (pgstop2),
 * conjugate gradient on the face until (cgstop1), projected search, and the
 * (cgstop3) switch; terminated by (bqp_approximate_sol). */
int ora_gpcg(const ora_stencil* A, const double* b, double c, const double* l,
             const double* u, const double* x0, const ora_options* opt, double* x,
             ora_stats* st, ora_event* events, int64_t event_cap, int64_t* event_len)
{
    const int64_t n = ora_n(A);
    const size_t bytes = sizeof(double) * (size_t)(n > 0 ? n : 1);
    double* g = (double*)malloc(bytes);
    double* w = (double*)malloc(bytes);
    uint8_t* act = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
    uint8_t* act_prev = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
    uint8_t* fr = (uint8_t*)malloc((size_t)(n > 0 ? n : 1));
    trace_t tr = {events, event_cap, 0};
    ora_census_out cs;
    int status = ORA_ERR_MAXIT;

    memset(st, 0, sizeof(*st));

    /* x0 in Omega: the given point projected, else l (Sec. 5 uses x0 = l),
     * falling back to u, then 0, where a bound is infinite. */
    for (int64_t i = 0; i < n; i++) {
        double xi;
        if (x0) xi = x0[i];
        else if (isfinite(l[i])) xi = l[i];
        else if (isfinite(u[i])) xi = u[i];
        else xi = 0.0;
        x[i] = mid(l[i], u[i], xi);
    }
    ora_census(A, b, c, l, u, x, g, act, &cs);
    const double pg0 = sqrt(cs.pg_norm2);
    const double tau = fmax(opt->tau_abs, opt->tau_rel * pg0);
    st->pg_norm0 = pg0;
    emit(&tr, ORA_EV_START, 0, 0, 0, cs.q, pg0, tau, 0.0);
    double pgn = pg0;
    if (pgn <= tau) {
        status = ORA_OK;
        goto finish;
    }

    double eta2 = opt->eta2;
    int continue_cg = 0;
    for (int k = 0; k < opt->max_outer; k++) {
        st->outer_iters = k + 1;
        if (!continue_cg) {
            /* gradient projection phase from y0 = x_k */
            double dmax = 0.0;
            for (int j = 1;; j++) {
                double alpha0 = 0.0, alpha = 0.0, decrease = 0.0;
                int trials = 0;
                memcpy(act_prev, act, (size_t)n);
                const int s = ora_gp_step(A, b, l, u, opt->mu, opt->max_ls, x, g,
                                          &alpha0, &alpha, &decrease, &trials);
                st->ls_trials += trials;
                if (s != ORA_OK) {
                    status = s;
                    goto finish;
                }
                st->gp_iters++;
                classify(n, b, c, l, u, x, g, act, &cs);
                pgn = sqrt(cs.pg_norm2);
                const int same = memcmp(act, act_prev, (size_t)n) == 0;
                emit(&tr, ORA_EV_GP_STEP, k, j, trials, alpha, decrease, same, pgn);
                if (pgn <= tau) {
                    status = ORA_OK;
                    goto finish;
                }
                int reason = 0;
                if (same) reason = ORA_GP_SAME_FACE;                              /* pgstop1 */
                else if (j >= 2 && decrease <= opt->eta1 * dmax) reason = ORA_GP_PROGRESS; /* pgstop2 */
                else if (j >= opt->max_gp) reason = ORA_GP_MAXIT;
                if (decrease > dmax) dmax = decrease;
                if (reason) {
                    emit(&tr, ORA_EV_GP_END, k, j, 0, reason, alpha0, 0.0, 0.0);
                    break;
                }
            }
        }
        /* conjugate gradient phase on the face of x_k */
        ORA_ROWS
        for (int64_t i = 0; i < n; i++) fr[i] = (uint8_t)!act[i];
        int iters = 0, reason = 0;
        int s = reduced_cg(A, fr, g, eta2, opt->max_cg, opt->precond, w, &iters, &reason, &tr,
                           k);
        st->cg_iters += iters;
        emit(&tr, ORA_EV_CG_END, k, iters, 0, reason, eta2, 0.0, 0.0);
        if (s != ORA_OK) {
            status = s;
            goto finish;
        }
        /* projected search along d_k = Z_k w */
        double alpha = 0.0, dq = 0.0;
        int trials = 0;
        s = ora_projected_search(A, b, l, u, opt->mu, opt->max_ls, w, x, g, &alpha,
                                 &dq, &trials);
        st->ls_trials += trials;
        if (s != ORA_OK) {
            status = s;
            goto finish;
        }
        classify(n, b, c, l, u, x, g, act, &cs);
        pgn = sqrt(cs.pg_norm2);
        const int bind_eq = cs.n_binding == cs.n_active; /* B subset of A */
        emit(&tr, ORA_EV_SEARCH, k, 0, trials, alpha, dq, pgn, bind_eq);
        if (pgn <= tau) {
            status = ORA_OK;
            goto finish;
        }
        if (bind_eq) { /* cgstop3: refine on the same face */
            eta2 = fmax(eta2 * opt->eta2_shrink, opt->eta2_floor);
            continue_cg = 1;
        } else {
            eta2 = opt->eta2;
            continue_cg = 0;
        }
    }

finish:
    ora_census(A, b, c, l, u, x, g, act, &cs);
    st->q = cs.q;
    st->pg_norm = sqrt(cs.pg_norm2);
    st->n_active = cs.n_active;
    st->n_binding = cs.n_binding;
    st->n_free = n - cs.n_active;
    st->status = status;
    emit(&tr, ORA_EV_DONE, st->outer_iters, 0, 0, status, st->pg_norm, st->q, 0.0);
    if (event_len) *event_len = tr.len;
    free(g);
    free(w);
    free(act);
    free(act_prev);
    free(fr);
    return status;
}
