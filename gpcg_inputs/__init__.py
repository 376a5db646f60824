"""Seeded synthetic inputs for GPCG: stencil Hessians, linear terms and bounds.

This module only *generates problems*; it holds none of the solver's
arithmetic.  Both the CPU oracle and the CUDA library receive the arrays it
returns, so the two sides always see bit-identical inputs.

Randomness is counter-based: every value is a pure function of
``(seed, stream, index)`` through the SplitMix64 output function (Steele, Lea &
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014), so a
problem is reproducible on any host and any slice of it can be regenerated
without the rest.

Problem family (the workloads of the GPCG paper are 2-D 5-point discretisations
with n up to 2.56e6, l = 0, u = +inf; the synthetic family below has the same
shapes and sparsity):

* A = L_w + s*I with L_w the weighted graph Laplacian of the grid graph whose
  edges carry weights w_e > 0, so A is symmetric positive definite with
  lambda_min(A) >= s.
* Band layout: ``diag[i] = A(i,i)``, ``cx[i] = A(i,i+1)``, ``cy[i] = A(i,i+nx)``,
  ``cz[i] = A(i,i+nx*ny)``, point ``i = ix + nx*(iy + ny*iz)``; the entry of the
  last point along an axis is stored as 0.

Workloads: the single small and single large QPs, the 512-instance batch, the
3-D precision-stress QP, the serving trace (Poisson arrivals; its requests
draw their QPs from a pool of log-spaced grid sizes), the journal bearing of
the paper's Sec. 5 and QPs whose solutions are free on a disc.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_STREAM = np.uint64(0xD1B54A32D192ED03)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (a bijection on 64-bit words)."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= np.uint64(0xBF58476D1CE4E5B9)
    z ^= z >> np.uint64(27)
    z *= np.uint64(0x94D049BB133111EB)
    z ^= z >> np.uint64(31)
    return z


def random_bits(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` 64-bit words for counter values ``offset .. offset+count-1``."""
    with np.errstate(over="ignore"):
        idx = np.arange(offset, offset + count, dtype=np.uint64) + np.uint64(1)
        base = _mix64(np.array([np.uint64(seed) ^ (np.uint64(stream) * _STREAM)],
                               dtype=np.uint64))[0]
        return _mix64(base + idx * _GOLDEN)


def uniform(seed: int, stream: int, count: int, lo: float = 0.0, hi: float = 1.0,
            offset: int = 0) -> np.ndarray:
    """Uniform doubles in [lo, hi) with 53 random bits each."""
    u = (random_bits(seed, stream, count, offset) >> np.uint64(11)).astype(np.float64)
    u *= 2.0 ** -53
    return lo + (hi - lo) * u


def normal(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """Standard normals by the Box-Muller transform of two uniform streams."""
    u1 = (random_bits(seed, 2 * stream, count, offset) >> np.uint64(11)).astype(np.float64)
    u1 = (u1 + 0.5) * 2.0 ** -53  # in (0, 1)
    u2 = uniform(seed, 2 * stream + 1, count, offset=offset)
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * math.pi * u2)


def lognormal(seed: int, stream: int, count: int, sigma: float, offset: int = 0) -> np.ndarray:
    return np.exp(sigma * normal(seed, stream, count, offset))


# Stream numbers, fixed so that one problem's parts never share random words.
_S_WX, _S_WY, _S_WZ, _S_B, _S_L, _S_U = 11, 12, 13, 21, 31, 32


@dataclass
class QP:
    """One bound-constrained QP  min 1/2 x'Ax + b'x + c,  l <= x <= u."""

    dim: int
    nx: int
    ny: int
    nz: int
    diag: np.ndarray
    cx: np.ndarray
    cy: np.ndarray
    cz: Optional[np.ndarray]
    b: np.ndarray
    l: np.ndarray
    u: np.ndarray
    c: float = 0.0
    shift: float = 0.0          # s in A = L_w + s I, a lower bound on lambda_min(A)
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.nx * self.ny * self.nz


def laplacian_bands_2d(nx: int, ny: int, wx: np.ndarray, wy: np.ndarray, shift: float):
    """Bands of A = L_w + shift*I for the nx-by-ny grid graph.

    ``wx`` (shape ny, nx-1) holds the weights of the edges (ix,iy)-(ix+1,iy) and
    ``wy`` (shape ny-1, nx) those of (ix,iy)-(ix,iy+1)."""
    cx = np.zeros((ny, nx))
    cy = np.zeros((ny, nx))
    cx[:, : nx - 1] = -wx
    cy[: ny - 1, :] = -wy
    deg = np.zeros((ny, nx))
    deg[:, : nx - 1] += wx
    deg[:, 1:] += wx
    deg[: ny - 1, :] += wy
    deg[1:, :] += wy
    return (deg + shift).ravel(), cx.ravel(), cy.ravel()


def laplacian_bands_3d(nx, ny, nz, wx, wy, wz, shift):
    """As :func:`laplacian_bands_2d` for an nx*ny*nz grid (arrays indexed [iz,iy,ix])."""
    cx = np.zeros((nz, ny, nx))
    cy = np.zeros((nz, ny, nx))
    cz = np.zeros((nz, ny, nx))
    cx[:, :, : nx - 1] = -wx
    cy[:, : ny - 1, :] = -wy
    cz[: nz - 1, :, :] = -wz
    deg = np.zeros((nz, ny, nx))
    deg[:, :, : nx - 1] += wx
    deg[:, :, 1:] += wx
    deg[:, : ny - 1, :] += wy
    deg[:, 1:, :] += wy
    deg[: nz - 1, :, :] += wz
    deg[1:, :, :] += wz
    return (deg + shift).ravel(), cx.ravel(), cy.ravel(), cz.ravel()


def grid_qp_2d(nx: int, ny: int, seed: int, shift: float, sigma: float = 0.5,
               bounds: str = "lower0", b_dist: str = "uniform", name: str = "") -> QP:
    """2-D 5-point QP: lognormal(0, sigma) edge weights, b ~ U[-1,1] (or N(0,1)).

    bounds: ``lower0`` (l = 0, u = +inf), ``two_sided`` (l ~ U[-0.5,0],
    u ~ U[0,0.5]), ``box1`` (l = -1, u = 1) or ``none`` (l = -inf, u = +inf)."""
    wx = lognormal(seed, _S_WX, ny * (nx - 1), sigma).reshape(ny, max(nx - 1, 0))
    wy = lognormal(seed, _S_WY, (ny - 1) * nx, sigma).reshape(max(ny - 1, 0), nx)
    diag, cx, cy = laplacian_bands_2d(nx, ny, wx, wy, shift)
    n = nx * ny
    b, l, u = _rhs_and_bounds(n, seed, bounds, b_dist)
    return QP(2, nx, ny, 1, diag, cx, cy, None, b, l, u, 0.0, shift, name or f"2d_{nx}x{ny}_s{seed}")


def grid_qp_3d(nx: int, ny: int, nz: int, seed: int, shift: float, sigma: float = 1.0,
               axis_scale=(1.0, 1.0, 1.0), bounds: str = "box1", b_dist: str = "normal",
               name: str = "") -> QP:
    """3-D 7-point QP: weights axis_scale[a] * lognormal(0, sigma) per axis."""
    wx = axis_scale[0] * lognormal(seed, _S_WX, nz * ny * (nx - 1), sigma)
    wy = axis_scale[1] * lognormal(seed, _S_WY, nz * (ny - 1) * nx, sigma)
    wz = axis_scale[2] * lognormal(seed, _S_WZ, (nz - 1) * ny * nx, sigma)
    diag, cx, cy, cz = laplacian_bands_3d(
        nx, ny, nz, wx.reshape(nz, ny, max(nx - 1, 0)), wy.reshape(nz, max(ny - 1, 0), nx),
        wz.reshape(max(nz - 1, 0), ny, nx), shift)
    n = nx * ny * nz
    b, l, u = _rhs_and_bounds(n, seed, bounds, b_dist)
    return QP(3, nx, ny, nz, diag, cx, cy, cz, b, l, u, 0.0, shift,
              name or f"3d_{nx}x{ny}x{nz}_s{seed}")


def _rhs_and_bounds(n: int, seed: int, bounds: str, b_dist: str):
    if b_dist == "uniform":
        b = uniform(seed, _S_B, n, -1.0, 1.0)
    elif b_dist == "normal":
        b = normal(seed, _S_B, n)
    else:
        raise ValueError(b_dist)
    if bounds == "lower0":
        l, u = np.zeros(n), np.full(n, np.inf)
    elif bounds == "two_sided":
        l, u = uniform(seed, _S_L, n, -0.5, 0.0), uniform(seed, _S_U, n, 0.0, 0.5)
    elif bounds == "box1":
        l, u = np.full(n, -1.0), np.full(n, 1.0)
    elif bounds == "none":
        l, u = np.full(n, -np.inf), np.full(n, np.inf)
    else:
        raise ValueError(bounds)
    return b, l, u


# --------------------------------------------------------------------------
# The five workloads.  Shapes follow the paper's benchmark (2-D 5-point,
# n = 1600^2 = 2.56e6); the journal-bearing discretisation itself is replaced
# by the weighted-Laplacian family above.
# --------------------------------------------------------------------------

def single_small() -> QP:
    """32x32 (n = 1024), shift 1e-2, b ~ U[-1,1], l = 0, u = +inf, seed 1."""
    return grid_qp_2d(32, 32, seed=1, shift=1e-2, bounds="lower0", name="single_32x32")


def single_large(side: int = 1600) -> QP:
    """1600x1600 (n = 2.56e6), shift 1e-3, two-sided bounds, seed 2."""
    return grid_qp_2d(side, side, seed=2, shift=1e-3, bounds="two_sided",
                      name=f"single_{side}x{side}")


def batch_sides(count: int = 512, seed: int = 3, lo: int = 64, hi: int = 512) -> np.ndarray:
    """Grid sides uniform on {lo..hi} for the batched workload."""
    u = uniform(seed, 1, count)
    return lo + np.floor(u * (hi - lo + 1)).astype(np.int64)


def batch_instance(k: int, side: int, seed: int = 3) -> QP:
    """Instance k of the batched workload: shift 1e-2, bounds one- or two-sided
    by a seeded coin."""
    coin = uniform(seed, 2, 1, offset=k)[0]
    bounds = "lower0" if coin < 0.5 else "two_sided"
    return grid_qp_2d(int(side), int(side), seed=1000 * seed + k, shift=1e-2, bounds=bounds,
                      name=f"batch{k}_{side}")


def precision_stress(side: int = 128) -> QP:
    """3-D 128^3 7-point, weights (1, 10, 100) x lognormal(0,1) per axis,
    shift 4 * max_axis_scale / 1e5, b ~ N(0,1), l = -1, u = 1, seed 4."""
    scale = (1.0, 10.0, 100.0)
    return grid_qp_3d(side, side, side, seed=4, shift=4.0 * max(scale) / 1e5, sigma=1.0,
                      axis_scale=scale, bounds="box1", b_dist="normal",
                      name=f"stress3d_{side}")


@dataclass
class Request:
    t_arrival: float
    dim: int
    side: int
    bounds: str
    seed: int


def serving_trace(rate: float = 200.0, duration: float = 60.0, seed: int = 5,
                  n_lo: float = 1e3, n_hi: float = 4e6) -> list:
    """Poisson arrivals; n log-uniform on [n_lo, n_hi]; 70% 2-D / 30% 3-D;
    bound type uniform over {lower0, two_sided, box1}."""
    out = []
    t = 0.0
    k = 0
    kinds = ("lower0", "two_sided", "box1")
    while True:
        u = uniform(seed, 1, 1, offset=k)[0]
        t += -math.log(1.0 - u) / rate
        if t >= duration:
            break
        un, ud, ub = uniform(seed, 2, 3, offset=3 * k)
        n = math.exp(math.log(n_lo) + un * (math.log(n_hi) - math.log(n_lo)))
        dim = 2 if ud < 0.7 else 3
        side = max(2, int(round(n ** (1.0 / dim))))
        out.append(Request(t, dim, side, kinds[min(int(ub * 3), 2)], 100000 * seed + k))
        k += 1
    return out


def serving_instance(r: Request) -> QP:
    if r.dim == 2:
        return grid_qp_2d(r.side, r.side, seed=r.seed, shift=1e-2, bounds=r.bounds,
                          name=f"req{r.seed}")
    return grid_qp_3d(r.side, r.side, r.side, seed=r.seed, shift=1e-2, sigma=0.5,
                      bounds=r.bounds, b_dist="uniform", name=f"req{r.seed}")


def serving_pool_sides(dim: int, count: int = 24, n_lo: float = 1e3, n_hi: float = 4e6) -> np.ndarray:
    """Grid sides of a size pool for the serving trace: n = side**dim
    log-spaced over [n_lo, n_hi] (duplicates after rounding removed)."""
    n = np.exp(np.linspace(math.log(n_lo), math.log(n_hi), count))
    return np.unique(np.maximum(2, np.round(n ** (1.0 / dim)).astype(np.int64)))


def pool_side(r: Request, sides: np.ndarray) -> int:
    """The pool side whose n is nearest to the request's in log scale."""
    k = int(np.argmin(np.abs(np.log(sides.astype(np.float64)) - math.log(r.side))))
    return int(sides[k])


def with_bounds(qp: QP, bounds: str, seed: int) -> QP:
    """The same Hessian and b with other bounds (arrays of A and b shared)."""
    if bounds == "lower0":
        l, u = np.zeros(qp.n), np.full(qp.n, np.inf)
    elif bounds == "two_sided":
        l, u = uniform(seed, _S_L, qp.n, -0.5, 0.0), uniform(seed, _S_U, qp.n, 0.0, 0.5)
    elif bounds == "box1":
        l, u = np.full(qp.n, -1.0), np.full(qp.n, 1.0)
    else:
        raise ValueError(bounds)
    return QP(qp.dim, qp.nx, qp.ny, qp.nz, qp.diag, qp.cx, qp.cy, qp.cz, qp.b, l, u, qp.c,
              qp.shift, f"{qp.name}_{bounds}")


def serving_pool(count: int = 24, seed: int = 6) -> dict:
    """Pre-generated QPs standing in for the serving trace's requests: for each
    dimension, the grids of :func:`serving_pool_sides` (shift 1e-2,
    lognormal(0, 0.5) weights, b ~ U[-1,1]), each with the three bound kinds of
    the trace.  Keys are (dim, side, bounds)."""
    pool = {}
    for dim in (2, 3):
        for k, side in enumerate(serving_pool_sides(dim, count)):
            s = int(side)
            ps = 1000 * seed + 100 * dim + k
            if dim == 2:
                base = grid_qp_2d(s, s, seed=ps, shift=1e-2, bounds="box1", name=f"pool2d_{s}")
            else:
                base = grid_qp_3d(s, s, s, seed=ps, shift=1e-2, sigma=0.5, bounds="box1",
                                  b_dist="uniform", name=f"pool3d_{s}")
            for kind in ("lower0", "two_sided", "box1"):
                pool[(dim, s, kind)] = base if kind == "box1" else with_bounds(base, kind, ps)
    return pool


def journal_bearing(nx: int, ny: int, eps: float, half_width: float = 10.0) -> QP:
    """The journal bearing problem of Sec. 5 as a finite-difference QP: minimise
    the integral of w_q |grad v|^2 / 2 - w_l v over D = (0, 2 pi) x (0, 2 b),
    w_q = (1 + eps cos xi_1)^3, w_l = eps sin xi_1, with v >= 0 and v = 0 on the
    boundary, on nx x ny interior points (h1 = 2 pi / (nx + 1), h2 = 2 b / (ny + 1),
    b = half_width).

    Each grid edge contributes w (v_i - v_j)^2 / 2 with w = w_q at the edge
    midpoint times h2/h1 (xi_1 edges) or h1/h2 (xi_2 edges); an edge to the
    boundary adds its w to the diagonal only (v = 0 there).  The linear term
    is b_i = -w_l(xi_1) h1 h2.  l = 0, u = +inf.  (The paper uses finite
    elements from a reference that is not at hand; this discretisation is
    for qualitative comparison only.)"""
    h1 = 2.0 * np.pi / (nx + 1)
    h2 = 2.0 * half_width / (ny + 1)
    wq = lambda t: (1.0 + eps * np.cos(t)) ** 3
    i = np.arange(1, nx + 1, dtype=np.float64)
    ax = wq((np.arange(0, nx + 1) + 0.5) * h1) * (h2 / h1)  # edge i+1/2, i = 0..nx
    cyw = wq(i * h1) * (h1 / h2)                            # xi_2 edges at column i
    diag_row = ax[:-1] + ax[1:] + 2.0 * cyw
    cx_row = np.zeros(nx)
    cx_row[:-1] = -ax[1:-1]
    diag = np.tile(diag_row, ny)
    cx = np.tile(cx_row, ny)
    cy = np.tile(-cyw, ny)
    cy[(ny - 1) * nx:] = 0.0
    b = np.tile(-eps * np.sin(i * h1) * h1 * h2, ny)
    n = nx * ny
    return QP(2, nx, ny, 1, diag, cx, cy, None, b, np.zeros(n), np.full(n, np.inf),
              shift=0.0, name=f"journal_bearing_{nx}x{ny}_eps{eps}",
              meta={"eps": eps, "half_width": half_width, "h1": h1, "h2": h2})


def disc_free_qp(side: int, free_frac: float, seed: int = 7, shift: float = 1e-2) -> QP:
    """A side x side QP whose solution is free on a disc covering about
    `free_frac` of the grid and at its lower bound elsewhere: the 5-point
    weighted Laplacian of grid_qp_2d, l = 0, u = +inf, b = -1 - |N(0,1)| / 4
    inside the disc (pulling x above 0) and +1 + |N(0,1)| / 4 outside (pressing
    it onto the bound).  For the masked-versus-extracted reduced system
    comparison across free fractions."""
    qp = grid_qp_2d(side, side, seed=seed, shift=shift, bounds="lower0",
                    name=f"disc_{side}_{free_frac}")
    iy, ix = np.divmod(np.arange(side * side), side)
    c = (side - 1) / 2.0
    rad = side * np.sqrt(free_frac / np.pi)
    inside = (ix - c) ** 2 + (iy - c) ** 2 <= rad * rad
    mag = 1.0 + np.abs(normal(seed, 11, side * side)) / 4.0
    qp.b = np.where(inside, -mag, mag)
    return qp
