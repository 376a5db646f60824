"""Brute-force solution of tiny bound-constrained QPs by enumerating faces.

TEST INFRASTRUCTURE ONLY (an independent pin for the oracle, not the oracle).

The feasible box Omega has at most 3^n faces (Sec. 5 of the GPCG paper); on
each face every variable sits at l_i, at u_i, or is free.  For a strictly
convex q the minimiser x* is unique (Sec. 2) and is the only point that
satisfies the Kuhn-Tucker conditions

    d_i q(x) = 0  if l_i < x_i < u_i,   >= 0  if x_i = l_i,   <= 0  if x_i = u_i.

For each face we solve A_FF x_F = -b_F - A_FA x_A by a Cholesky factorisation
and keep the candidate that is feasible and satisfies those sign conditions.
The dense matrix is assembled here edge by edge from the stencil bands, not
through the oracle's matrix-vector product.
"""
from __future__ import annotations

import itertools

import numpy as np


def dense_matrix(qp) -> np.ndarray:
    """Dense A from the bands: A[i,i] = diag[i]; A[i,j] = A[j,i] = c[i] for the
    east / north / up neighbour j of i along the band's axis."""
    n = qp.n
    A = np.zeros((n, n))
    nx, ny, nz = qp.nx, qp.ny, qp.nz
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                i = ix + nx * (iy + ny * iz)
                A[i, i] = qp.diag[i]
                if ix + 1 < nx:
                    A[i, i + 1] = A[i + 1, i] = qp.cx[i]
                if iy + 1 < ny:
                    A[i, i + nx] = A[i + nx, i] = qp.cy[i]
                if qp.dim == 3 and iz + 1 < nz:
                    A[i, i + nx * ny] = A[i + nx * ny, i] = qp.cz[i]
    return A


def kkt_residual(A, b, l, u, x):
    """Largest violation of feasibility and of the Kuhn-Tucker sign conditions."""
    g = A @ x + b
    viol = max(0.0, float(np.max(l - x, initial=0.0)), float(np.max(x - u, initial=0.0)))
    for i in range(x.size):
        at_l, at_u = x[i] == l[i], x[i] == u[i]
        if at_l and at_u:
            continue
        if at_l:
            viol = max(viol, -g[i])
        elif at_u:
            viol = max(viol, g[i])
        else:
            viol = max(viol, abs(g[i]))
    return viol


def solve_by_faces(qp, slack: float = 1e-12):
    """Return (x*, number of faces tried).  Raises if no or several distinct
    Kuhn-Tucker points are found."""
    A = dense_matrix(qp)
    b, l, u = np.asarray(qp.b, float), np.asarray(qp.l, float), np.asarray(qp.u, float)
    n = qp.n
    choices = []
    for i in range(n):
        opts = ["free"]
        if np.isfinite(l[i]):
            opts.append("l")
        if np.isfinite(u[i]) and u[i] != l[i]:
            opts.append("u")
        if l[i] == u[i]:
            opts = ["l"]
        choices.append(opts)
    found = []
    tried = 0
    scale = max(1.0, float(np.max(np.abs(A))), float(np.max(np.abs(b), initial=0.0)))
    for face in itertools.product(*choices):
        tried += 1
        x = np.zeros(n)
        free = np.array([f == "free" for f in face])
        for i, f in enumerate(face):
            if f == "l":
                x[i] = l[i]
            elif f == "u":
                x[i] = u[i]
        if free.any():
            F = np.flatnonzero(free)
            Af = A[np.ix_(F, F)]
            rhs = -b[F] - A[np.ix_(F, ~free)] @ x[~free]
            Lc = np.linalg.cholesky(Af)
            x[F] = np.linalg.solve(Lc.T, np.linalg.solve(Lc, rhs))
            # strictly inside the free range (else another face describes it)
            if np.any(x[F] < l[F] - slack * scale) or np.any(x[F] > u[F] + slack * scale):
                continue
        g = A @ x + b
        ok = True
        for i, f in enumerate(face):
            if f == "l" and l[i] != u[i] and g[i] < -slack * scale:
                ok = False
                break
            if f == "u" and g[i] > slack * scale:
                ok = False
                break
        if ok:
            found.append(x)
    if not found:
        raise RuntimeError("no Kuhn-Tucker point found")
    ref = found[0]
    for y in found[1:]:
        if np.max(np.abs(y - ref)) > 1e-8 * max(1.0, np.max(np.abs(ref))):
            raise RuntimeError("several distinct Kuhn-Tucker points")
    return np.clip(ref, l, u), tried
