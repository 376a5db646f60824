"""Thin ctypes binding of libgpcg.so (include/gpcg.h).

Argument marshalling only: every numerical step runs in the library's CUDA
kernels.  Arrays may be numpy arrays (host) or CUDA torch tensors (device);
both are passed to the C ABI as raw pointers.  Loading fails loudly when the
library is missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import _build

OK, ERR_ARG, ERR_INFEASIBLE, ERR_NUMERIC, ERR_OOM, ERR_BUDGET, ERR_CUDA = 0, 1, 2, 3, 4, 5, 6
ERR_MAXIT, ERR_LINESEARCH, ERR_TIMEOUT, ERR_PENDING, ERR_CANCELLED = 7, 8, 9, 10, 11
FP64, MIXED = 0, 1
PRECOND_NONE, PRECOND_JACOBI, PRECOND_TILE = 0, 1, 2
CG_MASKED, CG_EXTRACTED = 0, 1
PATH_AUTO, PATH_ENGINE, PATH_RESIDENT = 0, 1, 2

STATUS_NAMES = {0: "OK", 1: "ERR_ARG", 2: "ERR_INFEASIBLE", 3: "ERR_NUMERIC", 4: "ERR_OOM",
                5: "ERR_BUDGET", 6: "ERR_CUDA", 7: "ERR_MAXIT", 8: "ERR_LINESEARCH",
                9: "ERR_TIMEOUT", 10: "ERR_PENDING", 11: "ERR_CANCELLED"}


class GpcgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class gpcg_stencil(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64),
                ("diag", C.c_void_p), ("cx", C.c_void_p), ("cy", C.c_void_p),
                ("cz", C.c_void_p)]


class gpcg_options(C.Structure):
    _fields_ = [("tau_abs", C.c_double), ("tau_rel", C.c_double), ("eta1", C.c_double),
                ("eta2", C.c_double), ("mu", C.c_double), ("eta2_shrink", C.c_double),
                ("eta2_floor", C.c_double), ("max_outer", C.c_int), ("max_gp", C.c_int),
                ("max_cg", C.c_int), ("max_ls", C.c_int), ("precision", C.c_int),
                ("refine", C.c_int), ("x0", C.c_void_p), ("cuda_stream", C.c_void_p),
                ("lambda_min", C.c_double), ("precond", C.c_int), ("cg_system", C.c_int),
                ("path", C.c_int)]


_OPTION_FIELDS = frozenset(f for f, _ in gpcg_options._fields_)


class gpcg_stats(C.Structure):
    _fields_ = [("q", C.c_double), ("pg_norm", C.c_double), ("pg_norm0", C.c_double),
                ("tau", C.c_double), ("n_active", C.c_int64), ("n_binding", C.c_int64),
                ("n_free", C.c_int64), ("outer_iters", C.c_int), ("gp_iters", C.c_int),
                ("cg_iters", C.c_int), ("ls_trials", C.c_int), ("refine_cg_iters", C.c_int),
                ("passes", C.c_int), ("status", C.c_int), ("err_bound", C.c_double),
                ("alg_bytes", C.c_double), ("launches", C.c_int64), ("staged", C.c_int),
                ("fp64_gp_iters", C.c_int), ("mixed_n_active", C.c_int64),
                ("path", C.c_int), ("reserved", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None

# (name, restype, argtypes) for every entry point of include/gpcg.h
_SIGNATURES = [
    ("gpcg_problem_create", C.c_int, [C.POINTER(gpcg_stencil), C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_double, C.POINTER(C.c_void_p)]),
    ("gpcg_problem_update", C.c_int, [C.c_void_p, C.POINTER(gpcg_stencil), C.c_void_p,
                                      C.c_void_p, C.c_void_p, C.c_double]),
    ("gpcg_problem_update_async", C.c_int, [C.c_void_p, C.POINTER(gpcg_stencil), C.c_void_p,
                                            C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]),
    ("gpcg_problem_destroy", None, [C.c_void_p]),
    ("gpcg_problem_size", C.c_int64, [C.c_void_p]),
    ("gpcg_default_options", None, [C.POINTER(gpcg_options)]),
    ("gpcg_solve", C.c_int, [C.c_void_p, C.POINTER(gpcg_options)]),
    ("gpcg_solve_batch", C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.POINTER(gpcg_options)]),
    ("gpcg_result", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(gpcg_stats)]),
    ("gpcg_masked_spmv", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.POINTER(C.c_double), C.c_int, C.c_void_p]),
    ("gpcg_reduced_system", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.POINTER(C.c_int64),
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p]),
    ("gpcg_tile_precondition", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.POINTER(C.c_double), C.c_int, C.c_void_p]),
    ("gpcg_time_masked_spmv", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                        C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("gpcg_time_masked_spmv_stream", C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int,
                                               C.c_void_p, C.POINTER(C.c_double),
                                               C.POINTER(C.c_double)]),
    ("gpcg_masked_spmv_noalloc", C.c_int, [C.POINTER(gpcg_stencil), C.c_void_p, C.c_void_p,
                                           C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    ("gpcg_server_create", C.c_int, [C.c_size_t, C.c_int, C.POINTER(gpcg_options),
                                     C.POINTER(C.c_void_p)]),
    ("gpcg_server_submit", C.c_int, [C.c_void_p, C.POINTER(gpcg_stencil), C.c_void_p,
                                     C.c_void_p, C.c_void_p, C.c_double, C.c_void_p,
                                     C.POINTER(C.c_int64)]),
    ("gpcg_server_step", C.c_int, [C.c_void_p, C.c_int]),
    ("gpcg_server_done", C.c_int, [C.c_void_p, C.c_int64]),
    ("gpcg_server_stats", C.c_int, [C.c_void_p, C.c_int64, C.POINTER(gpcg_stats),
                                    C.POINTER(C.c_double)]),
    ("gpcg_server_cancel", C.c_int, [C.c_void_p, C.c_int64]),
    ("gpcg_server_timing", C.c_int, [C.c_void_p, C.POINTER(C.c_double)]),
    ("gpcg_server_counts", None, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_int)]),
    ("gpcg_server_destroy", None, [C.c_void_p]),
    ("gpcg_last_error", C.c_char_p, []),
    ("gpcg_version", C.c_char_p, []),
]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libgpcg.so (building it first if needed)."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libgpcg.so not found at {path}: build it with "
                               "paper_cs_0101018_gb300._build.build() (there is no CPU fallback)")
        L = C.CDLL(path)
        for name, res, args in _SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status):
    if status != OK:
        raise GpcgError(status, load().gpcg_last_error().decode())
    return status


def _ptr(a):
    """Raw pointer of a numpy array or a torch tensor (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _f64(a):
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float64)
    return a


def default_options(**kw) -> gpcg_options:
    o = gpcg_options()
    load().gpcg_default_options(C.byref(o))
    for k, v in kw.items():
        if k == "stream":
            k, v = "cuda_stream", (v.cuda_stream if hasattr(v, "cuda_stream") else v)
        if k == "x0":
            v = _ptr(v)
        if k not in _OPTION_FIELDS:
            raise TypeError(f"unknown gpcg option {k!r}")
        setattr(o, k, v)
    return o


class Problem:
    """A gpcg_problem handle plus the host/device arrays it was made from."""

    def __init__(self, handle, n, shape, dim=2):
        self.handle = handle
        self.n = n
        self.shape = shape
        self.dim = dim

    def __del__(self):
        try:
            if self.handle:
                load().gpcg_problem_destroy(self.handle)
                self.handle = None
        except Exception:
            pass


def _stencil(dim, nx, ny, nz, diag, cx, cy, cz):
    return gpcg_stencil(dim, nx, ny, nz, _ptr(diag), _ptr(cx), _ptr(cy), _ptr(cz))


def gpcg_problem_create(qp=None, *, dim=None, nx=None, ny=None, nz=1, diag=None, cx=None,
                        cy=None, cz=None, b=None, l=None, u=None, c=0.0) -> Problem:
    """Create a problem from a :class:`gpcg_inputs.QP` or from explicit arrays
    (numpy or CUDA tensors)."""
    if qp is not None:
        dim, nx, ny, nz = qp.dim, qp.nx, qp.ny, qp.nz
        diag, cx, cy, cz, b, l, u, c = qp.diag, qp.cx, qp.cy, qp.cz, qp.b, qp.l, qp.u, qp.c
    diag, cx, cy, cz, b, l, u = map(_f64, (diag, cx, cy, cz, b, l, u))
    st = _stencil(dim, nx, ny, nz, diag, cx, cy, cz)
    h = C.c_void_p()
    _check(load().gpcg_problem_create(C.byref(st), _ptr(b), _ptr(l), _ptr(u), float(c),
                                      C.byref(h)))
    return Problem(h, nx * ny * nz, (nx, ny, nz), dim)


def gpcg_problem_update(prob: Problem, qp=None, *, diag=None, cx=None, cy=None, cz=None, b=None,
                        l=None, u=None, c=0.0) -> None:
    """Replace the problem's data by a QP of the same grid (a
    :class:`gpcg_inputs.QP` or explicit arrays, numpy or CUDA tensors)."""
    nx, ny, nz = prob.shape
    dim = prob.dim
    if qp is not None:
        dim, nx, ny, nz = qp.dim, qp.nx, qp.ny, qp.nz
        diag, cx, cy, cz, b, l, u, c = qp.diag, qp.cx, qp.cy, qp.cz, qp.b, qp.l, qp.u, qp.c
    diag, cx, cy, cz, b, l, u = map(_f64, (diag, cx, cy, cz, b, l, u))
    st = _stencil(dim, nx, ny, nz, diag, cx, cy, cz)
    _check(load().gpcg_problem_update(prob.handle, C.byref(st), _ptr(b), _ptr(l), _ptr(u),
                                      float(c)))


def gpcg_problem_update_async(prob: Problem, qp=None, *, diag=None, cx=None, cy=None, cz=None,
                              b=None, l=None, u=None, c=0.0, stream=None) -> None:
    """gpcg_problem_update whose copies are only enqueued on `stream` (a
    torch.cuda.Stream, a raw handle or None); the next solve of the problem
    waits for them.  Pinned host arrays make the copies asynchronous; the
    problem keeps references to the arrays until its next update."""
    nx, ny, nz = prob.shape
    dim = prob.dim
    if qp is not None:
        dim, nx, ny, nz = qp.dim, qp.nx, qp.ny, qp.nz
        diag, cx, cy, cz, b, l, u, c = qp.diag, qp.cx, qp.cy, qp.cz, qp.b, qp.l, qp.u, qp.c
    diag, cx, cy, cz, b, l, u = map(_f64, (diag, cx, cy, cz, b, l, u))
    st = _stencil(dim, nx, ny, nz, diag, cx, cy, cz)
    sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(load().gpcg_problem_update_async(prob.handle, C.byref(st), _ptr(b), _ptr(l), _ptr(u),
                                            float(c), sp))
    prob.keep = (diag, cx, cy, cz, b, l, u, st)


def gpcg_solve(prob: Problem, opts: gpcg_options | None = None, check: bool = True) -> int:
    o = opts if opts is not None else default_options()
    s = load().gpcg_solve(prob.handle, C.byref(o))
    return _check(s) if check else s


def gpcg_solve_batch(probs, opts: gpcg_options | None = None, check: bool = True) -> int:
    o = opts if opts is not None else default_options()
    arr = (C.c_void_p * len(probs))(*[p.handle for p in probs])
    s = load().gpcg_solve_batch(arr, len(probs), C.byref(o))
    return _check(s) if check else s


def gpcg_result(prob: Problem, x_out=None):
    """Return (x, stats dict); x is written into x_out when given (numpy or
    CUDA tensor), else a new numpy array."""
    x = np.empty(prob.n) if x_out is None else x_out
    st = gpcg_stats()
    _check(load().gpcg_result(prob.handle, _ptr(x), C.byref(st)))
    return x, st.as_dict()


def gpcg_masked_spmv(prob: Problem, free_mask, p, precision=FP64, stream=None):
    """y = Z Z' A Z Z' p; returns (y, <p, Ap>)."""
    fm = np.ascontiguousarray(free_mask, dtype=np.uint8) if isinstance(free_mask, np.ndarray) \
        else free_mask
    p = _f64(p)
    y = np.empty(prob.n) if isinstance(p, np.ndarray) else p.new_empty(p.shape)
    pap = C.c_double()
    sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(load().gpcg_masked_spmv(prob.handle, _ptr(fm), _ptr(p), _ptr(y), C.byref(pap),
                                   precision, sp))
    return y, pap.value


def gpcg_reduced_system(prob: Problem, free_mask, dim=2, precision=FP64, stream=None):
    """The explicit reduced system for a free set: (m, fidx, diag, nb, val) with
    nb, val of shape (2*dim, m)."""
    fm = np.ascontiguousarray(free_mask, dtype=np.uint8)
    n = prob.n
    fidx = np.empty(n, np.int32)
    diag = np.empty(n)
    nb = np.empty(2 * dim * n, np.int32)
    val = np.empty(2 * dim * n)
    m = C.c_int64()
    sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(load().gpcg_reduced_system(prob.handle, _ptr(fm), precision, C.byref(m), _ptr(fidx),
                                      _ptr(diag), _ptr(nb), _ptr(val), sp))
    k = m.value
    return (k, fidx[:k].copy(), diag[:k].copy(), nb[:2 * dim * k].reshape(2 * dim, k).copy(),
            val[:2 * dim * k].reshape(2 * dim, k).copy())


def gpcg_tile_precondition(prob: Problem, free_mask, r, precision=FP64, stream=None):
    """z = M^-1 r of the tile preconditioner; returns (z, <r, z>)."""
    fm = np.ascontiguousarray(free_mask, dtype=np.uint8) if isinstance(free_mask, np.ndarray) \
        else free_mask
    r = _f64(r)
    z = np.empty(prob.n) if isinstance(r, np.ndarray) else r.new_empty(r.shape)
    rz = C.c_double()
    sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(load().gpcg_tile_precondition(prob.handle, _ptr(fm), _ptr(r), _ptr(z), C.byref(rz),
                                         precision, sp))
    return z, rz.value


def gpcg_time_masked_spmv(prob: Problem, precision=FP64, reps=20, flush_l2=True, stream=None):
    """(ms per launch, algorithmic bytes per launch) of the masked product."""
    ms, by = C.c_double(), C.c_double()
    sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    _check(load().gpcg_time_masked_spmv(prob.handle, precision, reps, int(bool(flush_l2)), sp,
                                        C.byref(ms), C.byref(by)))
    return ms.value, by.value


def gpcg_time_masked_spmv_stream(probs, precision=FP64, reps=10, stream=None):
    """(ms per launch, mean algorithmic bytes per launch) of the masked
    product in a stream of back-to-back launches over distinct problems."""
    ms, by = C.c_double(), C.c_double()
    sp = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    arr = (C.c_void_p * len(probs))(*[p.handle for p in probs])
    _check(load().gpcg_time_masked_spmv_stream(arr, len(probs), precision, reps, sp,
                                               C.byref(ms), C.byref(by)))
    return ms.value, by.value


@dataclass
class Ticket:
    id: int
    x: np.ndarray
    keep: tuple  # arrays that must stay alive until the request completes


class Server:
    """gpcg_server_*: continuous batching of independent solves."""

    def __init__(self, hbm_budget: int, max_live: int, opts: gpcg_options | None = None):
        o = opts if opts is not None else default_options()
        h = C.c_void_p()
        _check(load().gpcg_server_create(int(hbm_budget), int(max_live), C.byref(o), C.byref(h)))
        self.handle = h
        self.tickets = {}

    def submit(self, qp, x_out=None) -> Ticket:
        """Queue a QP (host arrays; pinned ones are copied by DMA without
        staging).  x_out: a float64 host array of n values for the solution
        (default: a new numpy array)."""
        arrs = tuple(np.ascontiguousarray(a, dtype=np.float64) if a is not None else None
                     for a in (qp.diag, qp.cx, qp.cy, qp.cz, qp.b, qp.l, qp.u))
        diag, cx, cy, cz, b, l, u = arrs
        st = _stencil(qp.dim, qp.nx, qp.ny, qp.nz, diag, cx, cy, cz)
        x = np.empty(qp.n) if x_out is None else x_out
        if x.dtype != np.float64 or x.size != qp.n or not x.flags["C_CONTIGUOUS"]:
            raise ValueError("x_out must be a contiguous float64 array of n values")
        t = C.c_int64()
        _check(load().gpcg_server_submit(self.handle, C.byref(st), _ptr(b), _ptr(l), _ptr(u),
                                         float(qp.c), _ptr(x), C.byref(t)))
        tk = Ticket(t.value, x, arrs + (st,))
        self.tickets[t.value] = tk
        return tk

    def step(self, passes: int = 32):
        _check(load().gpcg_server_step(self.handle, int(passes)))

    def done(self, tk: Ticket) -> bool:
        return bool(load().gpcg_server_done(self.handle, tk.id))

    def stats(self, tk: Ticket):
        st = gpcg_stats()
        lat = C.c_double()
        _check(load().gpcg_server_stats(self.handle, tk.id, C.byref(st), C.byref(lat)))
        return st.as_dict(), lat.value

    def release(self, tk: Ticket):
        """Drop the binding's references to a finished ticket's arrays (its x
        stays with the Ticket object)."""
        self.tickets.pop(tk.id, None)

    def cancel(self, tk: Ticket):
        _check(load().gpcg_server_cancel(self.handle, tk.id))

    def timing(self) -> dict:
        """Cumulative seconds of the server's step phases (gpcg_server_timing)."""
        v = (C.c_double * 8)()
        _check(load().gpcg_server_timing(self.handle, v))
        keys = ("admit_to_slots", "launch", "read_back", "start_uploads", "wait_passes",
                "device_passes", "steps", "steps_with_passes")
        return dict(zip(keys, list(v)))

    def counts(self):
        q, r, f = C.c_int(), C.c_int(), C.c_int()
        load().gpcg_server_counts(self.handle, C.byref(q), C.byref(r), C.byref(f))
        return q.value, r.value, f.value

    def close(self):
        if self.handle:
            load().gpcg_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
