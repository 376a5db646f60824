"""Python access to the FP64 CPU oracle (``gpcg_oracle.c``) for GPCG.

TEST INFRASTRUCTURE ONLY.  The test suite, the smoke check and the benchmark's
CPU-baseline leg use this package to produce the values the CUDA path is
compared against.  The CUDA library never imports, links or runs it, and it
imports nothing from the CUDA library: the two meet only in the seeded inputs
of :mod:`gpcg_inputs`.

The C code is built on first use with ``gcc -O2 -ffp-contract=off -fopenmp``
(every multiply and add separately rounded, identical on x86-64 and aarch64).
Loops whose rows are independent may run on several threads
(:func:`set_threads`); sums always run on one thread in index order, so
results do not depend on the thread count.  The default is one thread.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gpcg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_NUMERIC, ERR_MAXIT, ERR_LINESEARCH = 0, 3, 7, 8
EV_START, EV_GP_STEP, EV_GP_END, EV_CG_ITER, EV_CG_END, EV_SEARCH, EV_DONE = range(1, 8)
GP_SAME_FACE, GP_PROGRESS, GP_MAXIT = 1, 2, 3
CG_EMPTY, CG_PROGRESS, CG_EXACT, CG_MAXIT = 0, 1, 2, 3


class _Stencil(C.Structure):
    _fields_ = [("dim", C.c_int), ("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64),
                ("diag", C.c_void_p), ("cx", C.c_void_p), ("cy", C.c_void_p),
                ("cz", C.c_void_p)]


class Options(C.Structure):
    _fields_ = [("tau_abs", C.c_double), ("tau_rel", C.c_double), ("eta1", C.c_double),
                ("eta2", C.c_double), ("mu", C.c_double), ("eta2_shrink", C.c_double),
                ("eta2_floor", C.c_double), ("max_outer", C.c_int), ("max_gp", C.c_int),
                ("max_cg", C.c_int), ("max_ls", C.c_int), ("precond", C.c_int)]


class Stats(C.Structure):
    _fields_ = [("q", C.c_double), ("pg_norm", C.c_double), ("pg_norm0", C.c_double),
                ("n_active", C.c_int64), ("n_binding", C.c_int64), ("n_free", C.c_int64),
                ("outer_iters", C.c_int), ("gp_iters", C.c_int), ("cg_iters", C.c_int),
                ("ls_trials", C.c_int), ("status", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class _Census(C.Structure):
    _fields_ = [("n_active", C.c_int64), ("n_binding", C.c_int64), ("pg_norm2", C.c_double),
                ("q", C.c_double)]


class Event(C.Structure):
    _fields_ = [("kind", C.c_int), ("outer", C.c_int), ("inner", C.c_int),
                ("trials", C.c_int), ("a", C.c_double), ("b", C.c_double),
                ("c", C.c_double), ("d", C.c_double)]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (gcc, no CUDA)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
                os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "gpcg_oracle.h"))):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared",
                                   "-ffp-contract=off", "-fno-fast-math", "-fopenmp", _SRC,
                                   "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        vp, i64, dbl, ci = C.c_void_p, C.c_int64, C.c_double, C.c_int
        L.ora_set_threads.argtypes = [C.c_int]
        L.ora_set_threads.restype = None
        L.ora_get_threads.argtypes = []
        L.ora_get_threads.restype = C.c_int
        L.ora_set_threads(1)
        L.ora_default_options.argtypes = [C.POINTER(Options)]
        L.ora_matvec.argtypes = [C.POINTER(_Stencil), vp, vp]
        L.ora_masked_matvec.argtypes = [C.POINTER(_Stencil), vp, vp, vp]
        L.ora_q.argtypes = [C.POINTER(_Stencil), vp, dbl, vp]
        L.ora_q.restype = dbl
        L.ora_project.argtypes = [i64, vp, vp, vp, vp]
        L.ora_proj_gradient.argtypes = [i64, vp, vp, vp, vp, vp]
        L.ora_census.argtypes = [C.POINTER(_Stencil), vp, dbl, vp, vp, vp, vp, vp,
                                 C.POINTER(_Census)]
        L.ora_gp_step.argtypes = [C.POINTER(_Stencil), vp, vp, vp, dbl, ci, vp, vp,
                                  C.POINTER(dbl), C.POINTER(dbl), C.POINTER(dbl),
                                  C.POINTER(ci)]
        L.ora_gp_step.restype = ci
        L.ora_reduced_cg.argtypes = [C.POINTER(_Stencil), vp, vp, dbl, ci, ci, vp,
                                     C.POINTER(ci), C.POINTER(ci), vp, i64, C.POINTER(i64)]
        L.ora_reduced_cg.restype = ci
        L.ora_precondition.argtypes = [C.POINTER(_Stencil), vp, ci, vp, vp]
        L.ora_precondition.restype = None
        L.ora_projected_search.argtypes = [C.POINTER(_Stencil), vp, vp, vp, dbl, ci, vp, vp,
                                           vp, C.POINTER(dbl), C.POINTER(dbl), C.POINTER(ci)]
        L.ora_projected_search.restype = ci
        L.ora_gpcg.argtypes = [C.POINTER(_Stencil), vp, dbl, vp, vp, vp, C.POINTER(Options),
                               vp, C.POINTER(Stats), vp, i64, C.POINTER(i64)]
        L.ora_gpcg.restype = ci
        _lib = L
    return _lib


def set_threads(t: int) -> int:
    """Threads for the row loops (t <= 0: every processor); returns the count
    in force.  Results are bit-identical for every count."""
    lib().ora_set_threads(int(t))
    return int(lib().ora_get_threads())


def threads() -> int:
    return int(lib().ora_get_threads())


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class Stencil:
    """Holds the band arrays alive while the C struct points at them."""

    def __init__(self, qp):
        self.qp = qp
        self.diag, self.cx, self.cy = _f64(qp.diag), _f64(qp.cx), _f64(qp.cy)
        self.cz = _f64(qp.cz) if qp.dim == 3 else None
        self.s = _Stencil(qp.dim, qp.nx, qp.ny, qp.nz, _ptr(self.diag), _ptr(self.cx),
                          _ptr(self.cy), _ptr(self.cz))

    @property
    def ref(self):
        return C.byref(self.s)


def default_options(**kw) -> Options:
    o = Options()
    lib().ora_default_options(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def matvec(qp, x):
    st, x = Stencil(qp), _f64(x)
    y = np.empty_like(x)
    lib().ora_matvec(st.ref, _ptr(x), _ptr(y))
    return y


def masked_matvec(qp, free_mask, p):
    st, p = Stencil(qp), _f64(p)
    fm = np.ascontiguousarray(free_mask, dtype=np.uint8)
    y = np.empty_like(p)
    lib().ora_masked_matvec(st.ref, _ptr(fm), _ptr(p), _ptr(y))
    return y


def q_value(qp, x):
    st = Stencil(qp)
    return lib().ora_q(st.ref, _ptr(_f64(qp.b)), qp.c, _ptr(_f64(x)))


def project(l, u, x):
    l, u, x = _f64(l), _f64(u), _f64(x)
    out = np.empty_like(x)
    lib().ora_project(x.size, _ptr(l), _ptr(u), _ptr(x), _ptr(out))
    return out


def proj_gradient(x, g, l, u):
    x, g, l, u = _f64(x), _f64(g), _f64(l), _f64(u)
    out = np.empty_like(x)
    lib().ora_proj_gradient(x.size, _ptr(x), _ptr(g), _ptr(l), _ptr(u), _ptr(out))
    return out


@dataclass
class Census:
    g: np.ndarray
    active: np.ndarray
    n_active: int
    n_binding: int
    pg_norm2: float
    q: float


def census(qp, x) -> Census:
    st, x = Stencil(qp), _f64(x)
    b, l, u = _f64(qp.b), _f64(qp.l), _f64(qp.u)
    g = np.empty_like(x)
    act = np.empty(x.size, dtype=np.uint8)
    out = _Census()
    lib().ora_census(st.ref, _ptr(b), qp.c, _ptr(l), _ptr(u), _ptr(x), _ptr(g), _ptr(act),
                     C.byref(out))
    return Census(g, act.astype(bool), out.n_active, out.n_binding, out.pg_norm2, out.q)


def gp_step(qp, y, g, mu=0.01, max_ls=60):
    """One gradient projection iterate; returns (status, y', g', alpha0, alpha,
    decrease, trials)."""
    st = Stencil(qp)
    y, g = _f64(y).copy(), _f64(g).copy()
    a0, a, dec, tr = C.c_double(), C.c_double(), C.c_double(), C.c_int()
    s = lib().ora_gp_step(st.ref, _ptr(_f64(qp.b)), _ptr(_f64(qp.l)), _ptr(_f64(qp.u)), mu,
                          max_ls, _ptr(y), _ptr(g), C.byref(a0), C.byref(a), C.byref(dec),
                          C.byref(tr))
    return s, y, g, a0.value, a.value, dec.value, tr.value


PRECOND_NONE, PRECOND_JACOBI, PRECOND_TILE = 0, 1, 2
TILE_X, TILE_Y = 64, 8  # the blocks of PRECOND_TILE


def precondition(qp, free_mask, r, precond):
    """z = M^-1 r on the free set (zero elsewhere)."""
    st = Stencil(qp)
    fm = np.ascontiguousarray(free_mask, dtype=np.uint8)
    r = _f64(r)
    z = np.zeros_like(r)
    lib().ora_precondition(st.ref, _ptr(fm), precond, _ptr(r), _ptr(z))
    return z


def reduced_cg(qp, free_mask, g, eta2, max_cg, trace_cap=100000, precond=PRECOND_NONE):
    """(Preconditioned) CG on the reduced system from w0 = 0; returns (status, w,
    iters, reason, events); event c is <r_j, z_j> (= ||r_j||^2 without a
    preconditioner)."""
    st = Stencil(qp)
    fm = np.ascontiguousarray(free_mask, dtype=np.uint8)
    g = _f64(g)
    w = np.zeros_like(g)
    it, rs, ln = C.c_int(), C.c_int(), C.c_int64()
    ev = (Event * trace_cap)()
    s = lib().ora_reduced_cg(st.ref, _ptr(fm), _ptr(g), eta2, max_cg, precond, _ptr(w),
                             C.byref(it),
                             C.byref(rs), C.cast(ev, C.c_void_p), trace_cap, C.byref(ln))
    return s, w, it.value, rs.value, _events(ev, ln.value, trace_cap)


def projected_search(qp, x, g, d, mu=0.01, max_ls=60):
    st = Stencil(qp)
    x, g, d = _f64(x).copy(), _f64(g).copy(), _f64(d)
    a, dq, tr = C.c_double(), C.c_double(), C.c_int()
    s = lib().ora_projected_search(st.ref, _ptr(_f64(qp.b)), _ptr(_f64(qp.l)),
                                   _ptr(_f64(qp.u)), mu, max_ls, _ptr(d), _ptr(x), _ptr(g),
                                   C.byref(a), C.byref(dq), C.byref(tr))
    return s, x, g, a.value, dq.value, tr.value


def _events(ev, n, cap):
    return [dict(kind=e.kind, outer=e.outer, inner=e.inner, trials=e.trials, a=e.a, b=e.b,
                 c=e.c, d=e.d) for e in ev[: min(n, cap)]]


@dataclass
class Result:
    x: np.ndarray
    stats: dict
    events: list
    status: int


def solve(qp, x0=None, trace_cap: int = 0, **opts) -> Result:
    """Run Algorithm GPCG; ``opts`` override the default options by name."""
    st = Stencil(qp)
    o = default_options(**opts)
    x = np.empty(qp.n)
    stats = Stats()
    ev = (Event * max(trace_cap, 1))()
    ln = C.c_int64()
    x0a = _f64(x0) if x0 is not None else None
    s = lib().ora_gpcg(st.ref, _ptr(_f64(qp.b)), qp.c, _ptr(_f64(qp.l)), _ptr(_f64(qp.u)),
                       _ptr(x0a), C.byref(o), _ptr(x), C.byref(stats),
                       C.cast(ev, C.c_void_p) if trace_cap else None, trace_cap, C.byref(ln))
    return Result(x, stats.as_dict(), _events(ev, ln.value, trace_cap) if trace_cap else [], s)
