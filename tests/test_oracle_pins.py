"""Pins for the FP64 CPU oracle: each oracle function is checked against
something other than itself -- hand-derived closed forms, brute-force
enumeration of faces, dense linear algebra, textbook identities and the
invariants the GPCG paper states.  No GPU and no CUDA code is involved."""
import json
import math
import os

import numpy as np
import pytest

import gpcg_inputs as gi
import oracle
from oracle import brute_force as bf

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "kkt_closed_forms.json")


def _arr(v):
    return np.array([float(t) for t in v], dtype=np.float64)


def _golden_qp(case):
    n = case["nx"] * case["ny"] * case["nz"]
    return gi.QP(case["dim"], case["nx"], case["ny"], case["nz"], _arr(case["diag"]),
                 _arr(case["cx"]), _arr(case["cy"]),
                 _arr(case["cz"]) if case["dim"] == 3 else None, _arr(case["b"]),
                 _arr(case["l"]), _arr(case["u"]), float(case["c"]), 0.0, case["name"])


def _small_problems():
    """Tiny random problems covering 1-D chains, 2-D and 3-D grids, one- and
    two-sided bounds, infinite bounds and fixed variables."""
    out = []
    shapes2 = [(1, 1), (1, 6), (6, 1), (2, 3), (3, 3), (2, 4)]
    for k, (nx, ny) in enumerate(shapes2):
        for bounds in ("lower0", "two_sided", "box1"):
            qp = gi.grid_qp_2d(nx, ny, seed=100 + k, shift=0.05, bounds=bounds)
            out.append(qp)
    qp = gi.grid_qp_3d(2, 2, 2, seed=7, shift=0.05, sigma=0.5, bounds="two_sided",
                       b_dist="uniform")
    out.append(qp)
    # mixed infinite / fixed bounds
    qp = gi.grid_qp_2d(3, 3, seed=9, shift=0.05, bounds="two_sided")
    qp.l[0] = -np.inf
    qp.u[1] = np.inf
    qp.l[2] = qp.u[2] = 0.1
    qp.l[4], qp.u[4] = -np.inf, np.inf
    out.append(qp)
    return out


# ---------------------------------------------------------------------------
# matrix-vector product and the objective
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(1, 1), (7, 1), (1, 7), (5, 4), (13, 9)])
def test_matvec_matches_dense_assembly(shape):
    qp = gi.grid_qp_2d(*shape, seed=3, shift=0.1)
    A = bf.dense_matrix(qp)
    x = gi.uniform(5, 1, qp.n, -1, 1)
    y = oracle.matvec(qp, x)
    assert np.allclose(y, A @ x, rtol=0, atol=1e-13 * np.abs(A).sum(1).max())


@pytest.mark.parametrize("shape", [(1, 1, 1), (3, 1, 2), (4, 3, 2), (5, 5, 5)])
def test_matvec_3d_matches_dense_assembly(shape):
    qp = gi.grid_qp_3d(*shape, seed=4, shift=0.1, axis_scale=(1.0, 3.0, 9.0))
    A = bf.dense_matrix(qp)
    x = gi.normal(6, 1, qp.n)
    assert np.allclose(oracle.matvec(qp, x), A @ x, rtol=0,
                       atol=1e-13 * np.abs(A).sum(1).max())


def test_laplacian_quadratic_form():
    """x'(A - sI)x = sum over edges of w_e (x_i - x_j)^2 (graph Laplacian), and
    (A - sI) 1 = 0: pins the band convention independently of the dense
    assembly."""
    nx, ny, s = 6, 5, 0.25
    wx = gi.uniform(1, 1, ny * (nx - 1), 0.5, 2.0).reshape(ny, nx - 1)
    wy = gi.uniform(1, 2, (ny - 1) * nx, 0.5, 2.0).reshape(ny - 1, nx)
    diag, cx, cy = gi.laplacian_bands_2d(nx, ny, wx, wy, s)
    qp = gi.QP(2, nx, ny, 1, diag, cx, cy, None, np.zeros(nx * ny), np.zeros(nx * ny),
               np.zeros(nx * ny))
    x = gi.normal(2, 3, nx * ny)
    X = x.reshape(ny, nx)
    energy = (wx * (X[:, 1:] - X[:, :-1]) ** 2).sum() + (wy * (X[1:, :] - X[:-1, :]) ** 2).sum()
    Ax = oracle.matvec(qp, x)
    assert math.isclose(x @ Ax - s * (x @ x), energy, rel_tol=1e-12)
    assert np.allclose(oracle.matvec(qp, np.ones(nx * ny)), s, atol=1e-12)


def test_masked_matvec_is_reduced_hessian():
    qp = gi.grid_qp_2d(7, 6, seed=11, shift=0.1)
    A = bf.dense_matrix(qp)
    free = gi.uniform(3, 3, qp.n) < 0.6
    p = gi.normal(3, 4, qp.n)
    Z = np.eye(qp.n)[:, free]
    expect = Z @ (Z.T @ A @ Z) @ (Z.T @ p)
    assert np.allclose(oracle.masked_matvec(qp, free, p), expect, rtol=0, atol=1e-12)


def test_q_matches_definition():
    qp = gi.grid_qp_3d(3, 4, 2, seed=5, shift=0.2, bounds="box1")
    qp.c = -1.75
    A = bf.dense_matrix(qp)
    x = gi.uniform(8, 1, qp.n, -1, 1)
    assert math.isclose(oracle.q_value(qp, x), 0.5 * x @ A @ x + qp.b @ x + qp.c,
                        rel_tol=1e-13)


# ---------------------------------------------------------------------------
# projection, projected gradient, census
# ---------------------------------------------------------------------------

def test_projection_is_median_of_three():
    n = 2000
    l = gi.uniform(1, 1, n, -1, 0)
    u = gi.uniform(1, 2, n, 0, 1)
    l[:50], u[50:100], l[100:150] = -np.inf, np.inf, u[100:150]
    x = gi.normal(1, 3, n) * 2
    expect = np.median(np.stack([l, u, x]), axis=0)
    got = oracle.project(l, u, x)
    assert np.array_equal(got, expect)
    assert np.all((got >= l) & (got <= u))


def test_projected_gradient_is_limit_of_projected_step():
    """[grad_Omega q(x)]_i = lim_{t->0+} (x_i - P[x - t g]_i) / t, a
    characterisation independent of the case split (proj-gradient)."""
    n = 3000
    l = gi.uniform(2, 1, n, -1, 0)
    u = gi.uniform(2, 2, n, 0, 1)
    sel = gi.uniform(2, 3, n)
    x = l + (u - l) * gi.uniform(2, 4, n, 0.1, 0.9)  # free points well inside
    x = np.where(sel < 0.25, l, np.where(sel < 0.5, u, x))
    l[::97] = u[::97]
    x[::97] = l[::97]
    g = gi.normal(2, 5, n)
    t = 2.0 ** -24  # t*|g| stays far below the distance of free points to a bound
    lim = (x - oracle.project(l, u, x - t * g)) / t
    assert np.allclose(oracle.proj_gradient(x, g, l, u), lim, rtol=0, atol=1e-8)


def test_census_counts_and_values():
    qp = gi.grid_qp_2d(9, 7, seed=21, shift=0.1, bounds="two_sided")
    A = bf.dense_matrix(qp)
    sel = gi.uniform(21, 9, qp.n)
    x = np.where(sel < 0.3, qp.l, np.where(sel < 0.5, qp.u, 0.3 * qp.l + 0.7 * qp.u))
    c = oracle.census(qp, x)
    g = A @ x + qp.b
    assert np.allclose(c.g, g, atol=1e-13)
    at_l, at_u = x == qp.l, x == qp.u
    assert c.n_active == int(np.sum(at_l | at_u))
    assert c.n_binding == int(np.sum((at_l & (g >= 0)) | (at_u & (g <= 0))))
    assert np.array_equal(c.active, at_l | at_u)
    assert math.isclose(c.q, 0.5 * x @ A @ x + qp.b @ x, rel_tol=1e-12)
    pg = oracle.proj_gradient(x, g, qp.l, qp.u)
    assert math.isclose(c.pg_norm2, pg @ pg, rel_tol=1e-12)


# ---------------------------------------------------------------------------
# the gradient projection step, the reduced CG, the projected search
# ---------------------------------------------------------------------------

def _interior_point(qp, frac=0.4):
    sel = gi.uniform(77, 1, qp.n)
    lo = np.where(np.isfinite(qp.l), qp.l, -1.0)
    hi = np.where(np.isfinite(qp.u), qp.u, 1.0)
    return np.where(sel < frac, qp.l if np.all(np.isfinite(qp.l)) else lo, 0.5 * (lo + hi))


@pytest.mark.parametrize("bounds", ["two_sided", "lower0", "box1"])
def test_gp_step_alpha0_is_exact_line_minimiser(bounds):
    """alpha0 = argmin_{alpha>0} q(y - alpha grad_Omega q(y)) (bqpls): compare
    with a bounded scalar minimisation of the dense quadratic."""
    from scipy.optimize import minimize_scalar
    qp = gi.grid_qp_2d(8, 6, seed=31, shift=0.1, bounds=bounds)
    A = bf.dense_matrix(qp)
    y = oracle.project(qp.l, qp.u, _interior_point(qp))
    g = A @ y + qp.b
    pg = oracle.proj_gradient(y, g, qp.l, qp.u)
    s, y1, g1, a0, a, dec, trials = oracle.gp_step(qp, y, g)
    assert s == oracle.OK
    phi = lambda t: 0.5 * (y - t * pg) @ A @ (y - t * pg) + qp.b @ (y - t * pg)
    res = minimize_scalar(phi, bounds=(0, 10 * a0), method="bounded",
                          options={"xatol": 1e-12})
    assert math.isclose(a0, res.x, rel_tol=1e-5)
    assert phi(a0) <= phi(a0 * (1 + 1e-3)) and phi(a0) <= phi(a0 * (1 - 1e-3))


@pytest.mark.parametrize("seed", range(6))
def test_gp_step_sufficient_decrease_and_backtracking(seed):
    """The accepted point satisfies (gplsstop); the trial before it (twice the
    step) does not; the point is P[y - alpha g] (next-y); the reported decrease
    equals q(y) - q(y+) evaluated on the dense matrix."""
    qp = gi.grid_qp_2d(10, 9, seed=40 + seed, shift=0.02, bounds="two_sided")
    A = bf.dense_matrix(qp)
    q = lambda z: 0.5 * z @ A @ z + qp.b @ z
    y = oracle.project(qp.l, qp.u, np.zeros(qp.n) + 0.01 * seed)
    g = A @ y + qp.b
    mu = 0.3  # large mu forces some backtracking
    s, y1, g1, a0, a, dec, trials = oracle.gp_step(qp, y, g, mu=mu)
    assert s == oracle.OK
    assert a == a0 * 2.0 ** -(trials - 1)
    assert np.array_equal(y1, oracle.project(qp.l, qp.u, y - a * g))
    assert np.allclose(g1, A @ y1 + qp.b, atol=1e-13)
    scale = abs(q(y)) + 1
    assert math.isclose(dec, q(y) - q(y1), rel_tol=1e-9, abs_tol=1e-13 * scale)
    assert q(y1) <= q(y) + mu * g @ (y1 - y) + 1e-13 * scale
    if trials > 1:
        yp = oracle.project(qp.l, qp.u, y - 2 * a * g)
        assert q(yp) > q(y) + mu * g @ (yp - y) - 1e-13 * scale


def test_line_search_cap_gives_its_status():
    """With no backtracking allowed (max_ls = 0) and mu close to 1/2, a
    gradient-projection trial of this QP fails the sufficient-decrease test
    (Eq. gplsstop): the oracle stops in the GP phase with its line-search
    status at the last accepted point.  Recomputed here from the definitions
    (dense A, g = Ax + b, the projected gradient, alpha0 of Eq. bqpls and
    y = P[x - alpha0 g]), that trial violates the Armijo inequality.  With the
    default cap the same QP is solved."""
    qp = gi.grid_qp_2d(6, 5, seed=2, shift=0.01, sigma=1.5, bounds="two_sided")
    mu = 0.49
    r = oracle.solve(qp, tau_rel=1e-10, mu=mu, max_ls=0, trace_cap=1000)
    assert r.status == oracle.ERR_LINESEARCH
    assert r.events[-1]["kind"] == oracle.EV_DONE
    assert r.events[-2]["kind"] == oracle.EV_GP_STEP
    x = r.x
    assert np.all((x >= qp.l) & (x <= qp.u))
    A = bf.dense_matrix(qp)
    g = A @ x + qp.b
    pg = np.where(x <= qp.l, np.minimum(g, 0.0), np.where(x >= qp.u, np.maximum(g, 0.0), g))
    alpha0 = (pg @ pg) / (pg @ (A @ pg))
    y = np.minimum(np.maximum(x - alpha0 * g, qp.l), qp.u)
    q = lambda z: 0.5 * z @ (A @ z) + qp.b @ z
    assert q(y) > q(x) + mu * (g @ (y - x))
    assert oracle.solve(qp, tau_rel=1e-10, mu=mu).status == oracle.OK


def _lbfgsb_cases():
    out = [gi.grid_qp_2d(24, 20, seed=811, shift=0.05, bounds=b)
           for b in ("lower0", "two_sided", "box1")]
    out.append(gi.grid_qp_3d(8, 7, 6, seed=812, shift=0.05, sigma=0.5, bounds="box1"))
    return out


@pytest.mark.parametrize("case", range(4))
def test_gpcg_agrees_with_lbfgsb_within_certified_radii(case):
    """An independent algorithm (scipy's L-BFGS-B, a limited-memory
    quasi-Newton method with bounds) reaches the same unique minimiser, at
    sizes brute force cannot reach.  With r(x) = ||grad_Omega q(x)|| /
    lambda_min and lambda_min >= s, each point lies within r of x* (strong
    convexity), so ||x_gpcg - x_lbfgsb|| <= r(x_gpcg) + r(x_lbfgsb); the
    projected gradients are formed here from the definitions on dense A."""
    from scipy.optimize import minimize
    qp = _lbfgsb_cases()[case]
    A = bf.dense_matrix(qp)
    r = oracle.solve(qp, tau_rel=1e-12)
    assert r.status == oracle.OK

    def qg(x):
        g = A @ x + qp.b
        return 0.5 * x @ (A @ x) + qp.b @ x, g

    def radius(x):
        g = A @ x + qp.b
        pg = np.where(x <= qp.l, np.minimum(g, 0.0), np.where(x >= qp.u, np.maximum(g, 0.0), g))
        return float(np.linalg.norm(pg)) / qp.shift

    bounds = list(zip(np.where(np.isinf(qp.l), None, qp.l), np.where(np.isinf(qp.u), None, qp.u)))
    res = minimize(qg, np.clip(np.zeros(qp.n), qp.l, qp.u), jac=True, method="L-BFGS-B",
                   bounds=bounds, options=dict(maxiter=20000, ftol=1e-15, gtol=1e-12, maxcor=30))
    xl = np.clip(res.x, qp.l, qp.u)
    assert radius(xl) < 1e-4  # L-BFGS-B converged
    assert float(np.linalg.norm(xl - r.x)) <= radius(r.x) + radius(xl)
    assert radius(r.x) <= 1e-9


def test_reduced_cg_exact_solve_and_closed_form_decrease():
    """With eta2 = 0 the CG phase runs to the solution of A_FF w = -g_F (it
    terminates in at most m_k steps in exact arithmetic, Sec. 3); and the sum of
    the closed-form decreases Delta_j telescopes to q_k(0) - q_k(w)."""
    qp = gi.grid_qp_2d(9, 8, seed=50, shift=0.05)
    A = bf.dense_matrix(qp)
    free = gi.uniform(50, 2, qp.n) < 0.7
    g = gi.normal(50, 3, qp.n)
    s, w, iters, reason, ev = oracle.reduced_cg(qp, free, g, eta2=0.0, max_cg=4 * qp.n)
    assert s == oracle.OK
    F = np.flatnonzero(free)
    wF = np.linalg.solve(A[np.ix_(F, F)], -g[F])
    assert np.allclose(w[F], wF, rtol=1e-9, atol=1e-10)
    assert np.all(w[~free] == 0)
    qk = 0.5 * w[F] @ A[np.ix_(F, F)] @ w[F] + g[F] @ w[F]
    deltas = [e["b"] for e in ev if e["kind"] == oracle.EV_CG_ITER]
    assert math.isclose(sum(deltas), -qk, rel_tol=1e-10)
    assert all(e["d"] > 0 for e in ev if e["kind"] == oracle.EV_CG_ITER)


def _scaled_qp(qp):
    """The symmetrically scaled problem D^-1/2 A D^-1/2 (unit diagonal), built
    band by band: the couplings of points i and j divide by sqrt(d_i d_j)."""
    d = np.sqrt(qp.diag).reshape(qp.nz, qp.ny, qp.nx)
    cx = qp.cx.reshape(d.shape).copy()
    cy = qp.cy.reshape(d.shape).copy()
    cx[:, :, :-1] /= d[:, :, :-1] * d[:, :, 1:]
    cy[:, :-1, :] /= d[:, :-1, :] * d[:, 1:, :]
    return gi.QP(qp.dim, qp.nx, qp.ny, qp.nz, np.ones(qp.n), cx.ravel(), cy.ravel(), None,
                 qp.b, qp.l, qp.u)


def test_pcg_jacobi_exact_solve_and_closed_form_decrease():
    """Point-Jacobi PCG (Sec. 6) with eta2 = 0 reaches the solution of
    A_FF w = -g_F, and its closed-form decreases alpha_j rho_j / 2 telescope to
    q_k(0) - q_k(w)."""
    qp = gi.grid_qp_2d(9, 8, seed=56, shift=0.05, sigma=1.0)
    A = bf.dense_matrix(qp)
    free = gi.uniform(56, 2, qp.n) < 0.7
    g = gi.normal(56, 3, qp.n)
    s, w, iters, reason, ev = oracle.reduced_cg(qp, free, g, eta2=0.0, max_cg=4 * qp.n,
                                                precond=oracle.PRECOND_JACOBI)
    assert s == oracle.OK
    F = np.flatnonzero(free)
    AF = A[np.ix_(F, F)]
    wF = np.linalg.solve(AF, -g[F])
    assert np.allclose(w[F], wF, rtol=1e-9, atol=1e-10)
    assert np.all(w[~free] == 0)
    qk = 0.5 * w[F] @ AF @ w[F] + g[F] @ w[F]
    deltas = [e["b"] for e in ev if e["kind"] == oracle.EV_CG_ITER]
    assert math.isclose(sum(deltas), -qk, rel_tol=1e-10)


def test_pcg_jacobi_is_cg_on_the_scaled_system():
    """Jacobi PCG on A equals plain CG on D^-1/2 A D^-1/2 in the variables
    D^1/2 w: after any number of steps w = D^-1/2 w_hat, with the same alpha
    and the same rho (= ||r_hat||^2)."""
    qp = gi.grid_qp_2d(13, 11, seed=57, shift=0.02, sigma=1.0)
    sq = _scaled_qp(qp)
    free = gi.uniform(57, 2, qp.n) < 0.75
    g = gi.normal(57, 3, qp.n)
    dh = np.sqrt(qp.diag)
    for k in (1, 3, 7):
        s1, w, it1, _, ev1 = oracle.reduced_cg(qp, free, g, eta2=0.0, max_cg=k,
                                               precond=oracle.PRECOND_JACOBI)
        s2, wh, it2, _, ev2 = oracle.reduced_cg(sq, free, g / dh, eta2=0.0, max_cg=k)
        assert s1 == s2 == oracle.OK and it1 == it2 == k
        assert np.allclose(w, wh / dh, rtol=1e-10, atol=1e-13)
        a1 = [e["a"] for e in ev1 if e["kind"] == oracle.EV_CG_ITER]
        a2 = [e["a"] for e in ev2 if e["kind"] == oracle.EV_CG_ITER]
        c1 = [e["c"] for e in ev1 if e["kind"] == oracle.EV_CG_ITER]
        c2 = [e["c"] for e in ev2 if e["kind"] == oracle.EV_CG_ITER]
        assert np.allclose(a1, a2, rtol=1e-10) and np.allclose(c1, c2, rtol=1e-9)


def test_pcg_jacobi_special_cases():
    """Constant diagonal: Jacobi PCG takes exactly the CG steps (M is a
    multiple of I).  No couplings: the first step (alpha = 1) solves the
    diagonal system."""
    qp = gi.grid_qp_2d(10, 9, seed=58, shift=0.05)
    qp.diag[:] = 1.0 + float(np.max(qp.diag))  # constant, still diagonally dominant
    free = gi.uniform(58, 2, qp.n) < 0.8
    g = gi.normal(58, 3, qp.n)
    s1, w1, it1, r1, _ = oracle.reduced_cg(qp, free, g, eta2=0.05, max_cg=1000)
    s2, w2, it2, r2, _ = oracle.reduced_cg(qp, free, g, eta2=0.05, max_cg=1000,
                                           precond=oracle.PRECOND_JACOBI)
    assert (s1, it1, r1) == (s2, it2, r2)
    assert np.allclose(w1, w2, rtol=1e-12, atol=1e-15)
    qp.cx[:] = 0.0
    qp.cy[:] = 0.0
    # the first step is the solution (alpha = 1; the residual left is rounding)
    s, w, it, reason, ev = oracle.reduced_cg(qp, free, g, eta2=0.0, max_cg=1,
                                             precond=oracle.PRECOND_JACOBI)
    assert s == oracle.OK and it == 1
    assert math.isclose(ev[0]["a"], 1.0, rel_tol=1e-14)
    assert np.allclose(w[free], -g[free] / qp.diag[free], rtol=1e-14)
    assert ev[0]["c"] <= 1e-28 * np.sum(g[free] ** 2 / qp.diag[free])


def test_gpcg_with_jacobi_meets_the_same_tolerance():
    """GPCG with the Jacobi-preconditioned CG phase converges to the same
    minimiser (the KKT point is unique; only the path changes)."""
    qp = gi.grid_qp_2d(24, 20, seed=59, shift=0.02, bounds="two_sided", sigma=1.0)
    r0 = oracle.solve(qp, tau_rel=1e-11)
    r1 = oracle.solve(qp, tau_rel=1e-11, precond=oracle.PRECOND_JACOBI)
    assert r0.status == r1.status == oracle.OK
    assert r1.stats["pg_norm"] <= 1e-11 * r1.stats["pg_norm0"] * (1 + 1e-9)
    A = bf.dense_matrix(qp)
    assert bf.kkt_residual(A, qp.b, qp.l, qp.u, r1.x) < 1e-8
    assert np.allclose(r0.x, r1.x, rtol=1e-7, atol=1e-9)


def _tile_operator(qp, free):
    """M of the tile preconditioner on the free set, assembled densely from its
    definition: per 64 x 8 tile of each xy-plane, D = the couplings along x
    inside one row (the line tridiagonals, with the diagonal), L = the
    couplings from an odd row to an even row of the same tile, U = L',
    M = (D + L) D^-1 (D + U); nothing couples two tiles."""
    A = bf.dense_matrix(qp)
    F = np.flatnonzero(free)
    AF = A[np.ix_(F, F)]
    ix = F % qp.nx
    iy = (F // qp.nx) % qp.ny
    iz = F // (qp.nx * qp.ny)
    tile = (iz * 10**6 + (iy // oracle.TILE_Y)) * 10**6 + ix // oracle.TILE_X
    same_tile = tile[:, None] == tile[None, :]
    same_row = same_tile & (iy[:, None] == iy[None, :])
    odd_even = same_tile & (iy[:, None] % 2 == 1) & (iy[None, :] % 2 == 0)
    D = np.where(same_row, AF, 0.0)
    L = np.where(odd_even, AF, 0.0)
    return F, AF, (D + L) @ np.linalg.solve(D, D + L.T)


@pytest.mark.parametrize("case", ["2d", "3d", "ragged"])
def test_tile_preconditioner_is_the_zebra_operator(case):
    """The oracle's line sweeps (Thomas algorithm) apply exactly the inverse
    of the dense M = (D + L) D^-1 (D + U) of each tile."""
    if case == "2d":
        qp = gi.grid_qp_2d(70, 12, seed=60, shift=0.02, sigma=1.0)
    elif case == "3d":
        qp = gi.grid_qp_3d(66, 9, 3, seed=61, shift=0.02, sigma=0.5, bounds="two_sided",
                           b_dist="uniform")
    else:
        qp = gi.grid_qp_2d(131, 17, seed=62, shift=0.02, sigma=1.0)
    free = gi.uniform(60, 2, qp.n) < 0.7
    r = gi.normal(60, 3, qp.n)
    z = oracle.precondition(qp, free, r, oracle.PRECOND_TILE)
    F, _, M = _tile_operator(qp, free)
    assert np.all(z[~free] == 0.0)
    assert np.allclose(z[F], np.linalg.solve(M, r[F]), rtol=1e-11, atol=1e-13)


def test_tile_preconditioner_is_symmetric_positive_definite():
    """M^-1 (columns by applying it to unit vectors) is symmetric and positive
    definite, so PCG's theory holds."""
    qp = gi.grid_qp_2d(67, 10, seed=63, shift=0.02, sigma=1.0)
    free = gi.uniform(63, 2, qp.n) < 0.8
    F = np.flatnonzero(free)
    Z = np.empty((F.size, F.size))
    for k, i in enumerate(F):
        e = np.zeros(qp.n)
        e[i] = 1.0
        Z[:, k] = oracle.precondition(qp, free, e, oracle.PRECOND_TILE)[F]
    assert np.allclose(Z, Z.T, rtol=0, atol=1e-13 * np.max(np.abs(Z)))
    assert np.min(np.linalg.eigvalsh(0.5 * (Z + Z.T))) > 0.0


def test_pcg_tile_special_cases():
    """No couplings between rows and one tile column (nx <= 64): M = A_FF, so
    the first PCG step (alpha = 1) is the solution.  No couplings at all: the
    tile preconditioner is point Jacobi."""
    qp = gi.grid_qp_2d(60, 13, seed=64, shift=0.05, sigma=1.0)
    qp.cy[:] = 0.0
    free = gi.uniform(64, 2, qp.n) < 0.8
    g = gi.normal(64, 3, qp.n)
    s, w, it, reason, ev = oracle.reduced_cg(qp, free, g, eta2=0.0, max_cg=1,
                                             precond=oracle.PRECOND_TILE)
    A = bf.dense_matrix(qp)
    F = np.flatnonzero(free)
    assert s == oracle.OK and it == 1
    assert math.isclose(ev[0]["a"], 1.0, rel_tol=1e-13)
    assert np.allclose(w[F], np.linalg.solve(A[np.ix_(F, F)], -g[F]), rtol=1e-12, atol=1e-14)
    qp.cx[:] = 0.0
    r = gi.normal(64, 4, qp.n)
    zt = oracle.precondition(qp, free, r, oracle.PRECOND_TILE)
    zj = oracle.precondition(qp, free, r, oracle.PRECOND_JACOBI)
    assert np.array_equal(zt, zj)


def test_pcg_tile_exact_solve_and_closed_form_decrease():
    """Tile-preconditioned CG with eta2 = 0 reaches the solution of
    A_FF w = -g_F; its closed-form decreases telescope to q_k(0) - q_k(w); it
    needs fewer steps than point Jacobi on an anisotropic problem."""
    qp = gi.journal_bearing(70, 20, 0.5)
    A = bf.dense_matrix(qp)
    free = gi.uniform(65, 2, qp.n) < 0.85
    g = gi.normal(65, 3, qp.n)
    res = {}
    for pc in (oracle.PRECOND_JACOBI, oracle.PRECOND_TILE):
        s, w, iters, reason, ev = oracle.reduced_cg(qp, free, g, eta2=0.0, max_cg=4 * qp.n,
                                                    precond=pc)
        assert s == oracle.OK
        F = np.flatnonzero(free)
        AF = A[np.ix_(F, F)]
        assert np.allclose(w[F], np.linalg.solve(AF, -g[F]), rtol=1e-8, atol=1e-10)
        qk = 0.5 * w[F] @ AF @ w[F] + g[F] @ w[F]
        deltas = [e["b"] for e in ev if e["kind"] == oracle.EV_CG_ITER]
        assert math.isclose(sum(deltas), -qk, rel_tol=1e-9)
        res[pc] = iters
    assert res[oracle.PRECOND_TILE] < res[oracle.PRECOND_JACOBI]


def test_gpcg_with_tile_meets_the_same_tolerance():
    """GPCG with the tile-preconditioned CG phase reaches the same minimiser."""
    qp = gi.grid_qp_2d(90, 20, seed=66, shift=0.02, bounds="two_sided", sigma=1.0)
    r0 = oracle.solve(qp, tau_rel=1e-11)
    r1 = oracle.solve(qp, tau_rel=1e-11, precond=oracle.PRECOND_TILE)
    assert r0.status == r1.status == oracle.OK
    assert r1.stats["pg_norm"] <= 1e-11 * r1.stats["pg_norm0"] * (1 + 1e-9)
    A = bf.dense_matrix(qp)
    assert bf.kkt_residual(A, qp.b, qp.l, qp.u, r1.x) < 1e-8
    assert np.allclose(r0.x, r1.x, rtol=1e-7, atol=1e-9)


def test_reduced_cg_progress_stop():
    """(cgstop1): stop at the first j >= 2 with Delta_j <= eta2 max_{l<j} Delta_l
    and never earlier; the stopping step is included in w."""
    qp = gi.grid_qp_2d(30, 30, seed=51, shift=0.01)
    free = gi.uniform(51, 2, qp.n) < 0.8
    g = gi.normal(51, 3, qp.n)
    eta2 = 0.05
    s, w, iters, reason, ev = oracle.reduced_cg(qp, free, g, eta2=eta2, max_cg=10000)
    d = [e["b"] for e in ev if e["kind"] == oracle.EV_CG_ITER]
    assert reason == oracle.CG_PROGRESS and len(d) == iters
    for j in range(2, iters):
        assert d[j - 1] > eta2 * max(d[: j - 1])
    assert d[-1] <= eta2 * max(d[:-1])
    # w is the CG iterate after `iters` steps: compare with an independent
    # dense CG recurrence for the same number of steps
    A = bf.dense_matrix(qp)
    F = np.flatnonzero(free)
    AF = A[np.ix_(F, F)]
    r = g[F].copy()
    p = -r
    x = np.zeros(F.size)
    for _ in range(iters):
        Ap = AF @ p
        al = (r @ r) / (p @ Ap)
        x += al * p
        rn = r + al * Ap
        p = -rn + (rn @ rn) / (r @ r) * p
        r = rn
    assert np.allclose(w[F], x, rtol=1e-9, atol=1e-12)


def test_projected_search_first_unit_fraction():
    qp = gi.grid_qp_2d(12, 10, seed=60, shift=0.02, bounds="two_sided")
    A = bf.dense_matrix(qp)
    q = lambda z: 0.5 * z @ A @ z + qp.b @ z
    x = oracle.project(qp.l, qp.u, np.zeros(qp.n))
    g = A @ x + qp.b
    d = -4.0 * g  # an over-long descent direction forces backtracking
    s, x1, g1, a, dq, trials = oracle.projected_search(qp, x, g, d, mu=0.25)
    assert s == oracle.OK and trials >= 2
    assert a == 2.0 ** -(trials - 1)
    assert np.array_equal(x1, oracle.project(qp.l, qp.u, x + a * d))
    assert q(x1) <= q(x) + 0.25 * g @ (x1 - x) + 1e-12
    xp = oracle.project(qp.l, qp.u, x + 2 * a * d)
    assert q(xp) > q(x) + 0.25 * g @ (xp - x)
    assert math.isclose(dq, q(x1) - q(x), rel_tol=1e-9, abs_tol=1e-12)


# ---------------------------------------------------------------------------
# the whole algorithm
# ---------------------------------------------------------------------------

def test_golden_closed_forms():
    with open(GOLDEN) as f:
        cases = json.load(f)["cases"]
    for case in cases:
        qp = _golden_qp(case)
        r = oracle.solve(qp, tau_rel=0.0, tau_abs=1e-13)
        assert r.status == oracle.OK, case["name"]
        assert np.allclose(r.x, _arr(case["x_star"]), rtol=0, atol=1e-12), case["name"]
        assert math.isclose(r.stats["q"], float(case["q_star"]), rel_tol=1e-12,
                            abs_tol=1e-12), case["name"]
        # the brute-force enumerator agrees with the hand derivation too
        xb, _ = bf.solve_by_faces(qp)
        assert np.allclose(xb, _arr(case["x_star"]), atol=1e-12), case["name"]


@pytest.mark.parametrize("k", range(len(_small_problems())))
def test_gpcg_matches_brute_force(k):
    qp = _small_problems()[k]
    xs, faces = bf.solve_by_faces(qp)
    r = oracle.solve(qp, tau_rel=1e-13)
    assert r.status == oracle.OK
    A = bf.dense_matrix(qp)
    lam = np.linalg.eigvalsh(A)[0]
    # certified bound ||x - x*|| <= ||grad_Omega q(x)|| / lambda_min
    assert np.linalg.norm(r.x - xs) <= r.stats["pg_norm"] / lam * (1 + 1e-6) + 1e-12
    assert np.allclose(r.x, xs, atol=1e-9)
    assert bf.kkt_residual(A, qp.b, qp.l, qp.u, r.x) <= 1e-9
    assert np.all((r.x >= qp.l) & (r.x <= qp.u))


def test_gpcg_matches_brute_force_n12_one_sided():
    qp = gi.grid_qp_2d(4, 3, seed=123, shift=0.02, bounds="lower0")
    xs, faces = bf.solve_by_faces(qp)
    assert faces == 2 ** 12
    r = oracle.solve(qp, tau_rel=1e-13)
    assert r.status == oracle.OK
    assert np.allclose(r.x, xs, atol=1e-9)
    assert np.array_equal(r.x == 0.0, xs == 0.0)


def test_unconstrained_is_direct_solve():
    """With no finite bound, A(x) = B(x) = {} always, so after the first
    gradient projection phase (which stops on pgstop1 at j = 1) every outer
    iterate continues with CG (cgstop3), and x -> -A^{-1} b."""
    qp = gi.grid_qp_2d(15, 12, seed=70, shift=0.05, bounds="none")
    A = bf.dense_matrix(qp)
    r = oracle.solve(qp, tau_rel=1e-12, trace_cap=100000)
    assert r.status == oracle.OK
    xs = np.linalg.solve(A, -qp.b)
    assert np.allclose(r.x, xs, rtol=1e-9, atol=1e-9)
    gp_steps = [e for e in r.events if e["kind"] == oracle.EV_GP_STEP]
    assert len(gp_steps) == 1 and gp_steps[0]["c"] == 1.0
    assert all(e["d"] == 1.0 for e in r.events if e["kind"] == oracle.EV_SEARCH)


def test_diagonal_hessian_closed_form():
    """All couplings zero: x*_i = mid(l_i, u_i, -b_i / A_ii)."""
    n = 500
    qp = gi.grid_qp_2d(25, 20, seed=80, shift=0.5, bounds="two_sided")
    qp.cx[:] = 0.0
    qp.cy[:] = 0.0
    qp.diag[:] = gi.uniform(80, 7, n, 0.5, 3.0)
    r = oracle.solve(qp, tau_rel=1e-14)
    xs = np.median(np.stack([qp.l, qp.u, -qp.b / qp.diag]), axis=0)
    assert r.status == oracle.OK
    assert np.allclose(r.x, xs, atol=1e-13)


def _check_trace_invariants(qp, r, eta1=0.1, eta2=0.05, shrink=0.1, mu=0.01):
    ev = r.events
    assert ev[0]["kind"] == oracle.EV_START and ev[-1]["kind"] == oracle.EV_DONE
    tau = ev[0]["c"]
    assert r.status == oracle.OK and r.stats["pg_norm"] <= tau
    assert np.all((r.x >= qp.l) & (r.x <= qp.u))
    # gradient projection phases: decreases positive, stop rules as defined
    phase = []
    eta2_now = eta2
    expect_gp = True
    for e in ev:
        if e["kind"] == oracle.EV_GP_STEP:
            assert expect_gp
            assert e["b"] > 0  # q strictly decreases at an accepted GP step
            phase.append(e)
        elif e["kind"] == oracle.EV_GP_END:
            decs = [p["b"] for p in phase]
            j = len(phase)
            for i in range(1, j):  # no stop rule held before the last step
                assert phase[i - 1]["c"] == 0.0
                if i >= 2:
                    assert decs[i - 1] > eta1 * max(decs[: i - 1])
            last = phase[-1]
            stop1 = last["c"] == 1.0
            stop2 = j >= 2 and decs[-1] <= eta1 * max(decs[:-1])
            assert stop1 or stop2 or j >= 50
            phase = []
        elif e["kind"] == oracle.EV_CG_END:
            assert e["b"] == pytest.approx(eta2_now, rel=1e-15)
        elif e["kind"] == oracle.EV_CG_ITER:
            assert e["d"] > 0 and e["b"] > 0
        elif e["kind"] == oracle.EV_SEARCH:
            assert e["b"] <= 0  # q(x_{k+1}) <= q(x_k)
            if e["d"] == 1.0:
                eta2_now = max(eta2_now * shrink, 1e-12)
                expect_gp = False
            else:
                eta2_now = eta2
                expect_gp = True


@pytest.mark.parametrize("bounds", ["lower0", "two_sided", "box1"])
def test_trace_invariants(bounds):
    qp = gi.grid_qp_2d(40, 30, seed=90, shift=0.01, bounds=bounds)
    r = oracle.solve(qp, tau_rel=1e-10, trace_cap=200000)
    _check_trace_invariants(qp, r)


def test_trace_invariants_3d():
    qp = gi.grid_qp_3d(10, 9, 8, seed=91, shift=0.01, sigma=0.5, axis_scale=(1, 10, 100))
    r = oracle.solve(qp, tau_rel=1e-9, trace_cap=400000)
    _check_trace_invariants(qp, r)


def test_single_small_workload_solution_is_kkt():
    qp = gi.single_small()
    r = oracle.solve(qp, tau_rel=1e-8)
    assert r.status == oracle.OK
    A = bf.dense_matrix(qp)
    xs = np.clip(r.x, qp.l, qp.u)
    assert np.array_equal(xs, r.x)
    lam = np.linalg.eigvalsh(A)[0]
    assert lam >= qp.shift * (1 - 1e-12)
    assert bf.kkt_residual(A, qp.b, qp.l, qp.u, r.x) <= r.stats["pg_norm"] * 1.000001
