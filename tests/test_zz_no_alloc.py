"""The allocation-free masked product (gpcg_masked_spmv_noalloc) against the
regular one (gpcg_masked_spmv, FP64) and against the oracle's masked product,
through the C ABI.

This entry point serves callers that cannot allocate device memory (their
device memory belongs to their own pool allocator, or they run in loops that
cannot take the synchronisation cudaMalloc may cause); its only scratch is a
fixed array inside the library.  This file is collected last so that a run
stopping at the first failure has already run every other test; it also
passes on its own in a fresh process."""
import ctypes as C

import numpy as np
import pytest

import gpcg_inputs as gi
import oracle

g = pytest.importorskip("paper_cs_0101018_gb300")
from paper_cs_0101018_gb300.gpcg import gpcg_stencil  # noqa: E402

pytestmark = pytest.mark.gpu

EPS64 = np.finfo(np.float64).eps


def _abs_a_abs_p(qp, fm, p):
    """(|A_FF| |p_F|) on the free set, from the bands (the error scale of a
    stencil row sum of at most 7 terms)."""
    nx, ny, nz = qp.nx, qp.ny, qp.nz
    pa = np.abs(p * fm).reshape(nz, ny, nx)
    out = np.abs(qp.diag).reshape(nz, ny, nx) * pa
    cx, cy = np.abs(qp.cx).reshape(nz, ny, nx), np.abs(qp.cy).reshape(nz, ny, nx)
    out[:, :, :-1] += cx[:, :, :-1] * pa[:, :, 1:]
    out[:, :, 1:] += cx[:, :, :-1] * pa[:, :, :-1]
    out[:, :-1, :] += cy[:, :-1, :] * pa[:, 1:, :]
    out[:, 1:, :] += cy[:, :-1, :] * pa[:, :-1, :]
    if qp.dim == 3:
        cz = np.abs(qp.cz).reshape(nz, ny, nx)
        out[:-1] += cz[:-1] * pa[1:]
        out[1:] += cz[:-1] * pa[:-1]
    return out.ravel() * fm


@pytest.mark.parametrize("shape", [(1, 1, 1), (200, 97, 1), (1600, 1600, 1), (33, 17, 5)])
def test_noalloc_matches_masked_spmv(shape):
    import torch
    nx, ny, nz = shape
    qp = (gi.grid_qp_2d(nx, ny, seed=11, shift=0.1) if nz == 1 else
          gi.grid_qp_3d(nx, ny, nz, seed=11, shift=0.1, axis_scale=(1, 10, 100)))
    fm = gi.uniform(12, 1, qp.n) < 0.6
    p = gi.normal(12, 2, qp.n)
    prob = g.gpcg_problem_create(qp)
    y_ref, pap_ref = g.gpcg_masked_spmv(prob, fm, p, precision=g.FP64)
    y_ora = oracle.masked_matvec(qp, fm, p)
    pap_ora = float(np.dot(p[fm], y_ora[fm]))

    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    bands = [dev(qp.diag), dev(qp.cx), dev(qp.cy), dev(qp.cz) if nz > 1 else None]
    st = gpcg_stencil(qp.dim, nx, ny, nz, *[b.data_ptr() if b is not None else None
                                            for b in bands])
    d_fm = dev(fm.astype(np.uint8))
    d_p = dev(p)
    bound = _abs_a_abs_p(qp, fm, p)
    L = g.load()
    for call in range(2):  # two calls in a row share the scratch array
        d_y = torch.full((qp.n,), np.nan, dtype=torch.float64, device="cuda")
        pap = C.c_double(np.nan)
        s = L.gpcg_masked_spmv_noalloc(C.byref(st), d_fm.data_ptr(), d_p.data_ptr(),
                                       d_y.data_ptr(), C.byref(pap), None)
        assert s == g.OK, L.gpcg_last_error()
        y = d_y.cpu().numpy()
        assert np.all(np.abs(y - y_ref) <= 16 * EPS64 * bound + 1e-300), call
        assert np.all(np.abs(y - y_ora) <= 8 * EPS64 * bound + 1e-300), call
        assert np.all(y[~fm] == 0.0)
        assert np.isclose(pap.value, pap_ref, rtol=1e-12, atol=1e-300), (call, pap.value, pap_ref)
        assert np.isclose(pap.value, pap_ora, rtol=1e-12, atol=1e-300), (call, pap.value, pap_ora)


def test_noalloc_rejects_what_it_cannot_serve():
    import torch
    L = g.load()
    nx = ny = 4096  # 64 x 128 tiles = 8192 > the 4096-tile scratch
    one = torch.ones(1, dtype=torch.float64, device="cuda")
    st = gpcg_stencil(2, nx, ny, 1, one.data_ptr(), one.data_ptr(), one.data_ptr(), None)
    assert L.gpcg_masked_spmv_noalloc(C.byref(st), one.data_ptr(), one.data_ptr(),
                                      one.data_ptr(), None, None) == g.ERR_ARG
    assert b"too large" in L.gpcg_last_error()
    # y must not overlap an input: neighbouring CTAs still read p where y is written
    qp = gi.grid_qp_2d(40, 30, seed=13, shift=0.1)
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    bands = [dev(qp.diag), dev(qp.cx), dev(qp.cy)]
    st = gpcg_stencil(2, qp.nx, qp.ny, 1, *[b.data_ptr() for b in bands], None)
    d_fm = dev(np.ones(qp.n, dtype=np.uint8))
    d_p = dev(gi.normal(13, 1, qp.n))
    assert L.gpcg_masked_spmv_noalloc(C.byref(st), d_fm.data_ptr(), d_p.data_ptr(),
                                      d_p.data_ptr(), None, None) == g.ERR_ARG
    assert b"overlap" in L.gpcg_last_error()
    assert L.gpcg_masked_spmv_noalloc(C.byref(st), d_fm.data_ptr(), d_p.data_ptr(),
                                      bands[0].data_ptr() + 8, None, None) == g.ERR_ARG
    host = np.ones(16)
    st = gpcg_stencil(2, 4, 4, 1, host.ctypes.data, host.ctypes.data, host.ctypes.data, None)
    assert L.gpcg_masked_spmv_noalloc(C.byref(st), host.ctypes.data, host.ctypes.data,
                                      host.ctypes.data, None, None) == g.ERR_ARG
