"""CPU-only checks of the C ABI: the library builds, loads, exports every
symbol include/gpcg.h declares, and rejects bad arguments before touching the
GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "gpcg.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gpcg_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_entry_points():
    names = _declared()
    for must in ("gpcg_problem_create", "gpcg_solve", "gpcg_result", "gpcg_solve_batch",
                 "gpcg_masked_spmv", "gpcg_server_create", "gpcg_server_submit"):
        assert must in names


def test_library_exports_every_declared_symbol():
    import paper_cs_0101018_gb300 as g
    L = g.load()
    for name in _declared():
        assert hasattr(L, name), name
    assert b"sm_103a" in L.gpcg_version()


def test_python_binding_covers_every_symbol():
    from paper_cs_0101018_gb300 import gpcg
    bound = {n for n, _, _ in gpcg._SIGNATURES}
    assert set(_declared()) <= bound


def test_default_options_are_the_papers():
    import paper_cs_0101018_gb300 as g
    o = g.default_options()
    assert (o.eta1, o.eta2) == (0.1, 0.05)     # Sec. 5
    assert 0 < o.mu < 0.5                      # Eq. gplsstop asks mu in (0, 1/2)
    assert o.precision == g.FP64 and o.refine == 2 and o.path == g.PATH_AUTO


def test_argument_checks_need_no_gpu():
    import paper_cs_0101018_gb300 as g
    L = g.load()
    from paper_cs_0101018_gb300.gpcg import gpcg_stencil, gpcg_options
    out = C.c_void_p()
    # NULL stencil / bad dimensions are rejected before any CUDA call
    assert L.gpcg_problem_create(None, None, None, None, 0.0, C.byref(out)) == g.ERR_ARG
    st = gpcg_stencil(4, 2, 2, 1, None, None, None, None)
    assert L.gpcg_problem_create(C.byref(st), None, None, None, 0.0, C.byref(out)) == g.ERR_ARG
    st = gpcg_stencil(2, 2, 2, 3, None, None, None, None)
    assert L.gpcg_problem_create(C.byref(st), None, None, None, 0.0, C.byref(out)) == g.ERR_ARG
    assert b"" != L.gpcg_last_error()
    o = g.default_options(mu=0.7)
    assert L.gpcg_solve(None, C.byref(o)) == g.ERR_ARG
    srv = C.c_void_p()
    assert L.gpcg_server_create(0, 4, C.byref(o), C.byref(srv)) == g.ERR_ARG
    o = g.default_options(mu=0.7)
    assert L.gpcg_server_create(1 << 30, 4, C.byref(o), C.byref(srv)) == g.ERR_ARG
    # options are checked before any CUDA call: unknown preconditioner or CG
    # system, and the tile preconditioner with the extracted reduced system
    for bad in (dict(precond=3), dict(cg_system=2),
                dict(precond=g.PRECOND_TILE, cg_system=g.CG_EXTRACTED)):
        o = g.default_options(**bad)
        assert L.gpcg_server_create(1 << 30, 4, C.byref(o), C.byref(srv)) == g.ERR_ARG


def test_option_defaults_are_the_masked_unpreconditioned_cg():
    import paper_cs_0101018_gb300 as g
    o = g.default_options()
    assert o.precond == g.PRECOND_NONE and o.cg_system == g.CG_MASKED


def test_oracle_and_library_share_no_code():
    """The oracle (C, gcc) and the CUDA library must not include each other."""
    csrc = os.path.join(ROOT, "paper_cs_0101018_gb300", "csrc")
    for fn in os.listdir(csrc):
        with open(os.path.join(csrc, fn)) as f:
            assert "oracle" not in f.read().lower(), fn
    for fn in ("gpcg_oracle.c", "gpcg_oracle.h", "__init__.py", "brute_force.py"):
        with open(os.path.join(ROOT, "oracle", fn)) as f:
            txt = f.read()
        assert "paper_cs_0101018_gb300" not in txt and "csrc" not in txt, fn


def test_update_and_server_calls_reject_bad_arguments_without_a_gpu():
    import paper_cs_0101018_gb300 as g
    L = g.load()
    from paper_cs_0101018_gb300.gpcg import gpcg_stencil
    st = gpcg_stencil(2, 4, 4, 1, None, None, None, None)
    # NULL problem handle: rejected before any CUDA call
    assert L.gpcg_problem_update(None, C.byref(st), None, None, None, 0.0) == g.ERR_ARG
    assert L.gpcg_problem_update_async(None, C.byref(st), None, None, None, 0.0,
                                       None) == g.ERR_ARG
    v = (C.c_double * 8)()
    assert L.gpcg_server_timing(None, v) == g.ERR_ARG
    assert L.gpcg_server_step(None, 16) == g.ERR_ARG
    assert L.gpcg_server_cancel(None, 1) == g.ERR_ARG
    assert L.gpcg_server_done(None, 1) == 0
    t = C.c_int64()
    assert L.gpcg_server_submit(None, C.byref(st), None, None, None, 0.0, None,
                                C.byref(t)) == g.ERR_ARG


def test_size_limit_is_checked_before_any_copy():
    """The padded count px*ny*nz (px = nx rounded up to 8) must stay below
    2^31: larger problems are refused with GPCG_ERR_ARG before any array is
    read, also where the plain product nx*ny*nz would wrap around (to 0 for
    (2^22, 2^22, 2^20)) or where padding nx would leave the int range."""
    import numpy as np
    import paper_cs_0101018_gb300 as g
    from paper_cs_0101018_gb300.gpcg import gpcg_stencil
    L = g.load()
    dummy = np.zeros(4)
    p = dummy.ctypes.data
    out = C.c_void_p()
    for dims in ((2, 1 << 16, 1 << 16, 1), (3, 1 << 11, 1 << 10, 1 << 10), (2, 1 << 31, 1, 1),
                 (3, 1 << 22, 1 << 22, 1 << 20), (2, (1 << 31) - 1, 1, 1),
                 (2, (1 << 31) - 8, 1, 1), (2, 1, 1 << 28, 1), (3, 8, 1 << 14, 1 << 14),
                 (3, 1 << 62, 1 << 2, 1 << 0)):
        st = gpcg_stencil(dims[0], dims[1], dims[2], dims[3], p, p, p, p)
        assert L.gpcg_problem_create(C.byref(st), p, None, None, 0.0, C.byref(out)) == g.ERR_ARG
        assert b"too large" in L.gpcg_last_error()


def test_noalloc_size_limit_is_checked_before_any_cuda_call():
    """The allocation-free product refuses grids beyond its fixed scratch
    (4096 tiles of 64x32 points) and extents whose tile product would wrap,
    before it asks CUDA anything."""
    import numpy as np
    import paper_cs_0101018_gb300 as g
    from paper_cs_0101018_gb300.gpcg import gpcg_stencil
    L = g.load()
    dummy = np.zeros(4)
    p = dummy.ctypes.data
    for dims in ((2, 4096, 4096, 1), (2, 1 << 31, 1, 1), (3, 1 << 40, 1 << 40, 1 << 40),
                 (3, 64, 32, 4097), (3, 1 << 21, 1 << 21, 1 << 22)):
        st = gpcg_stencil(dims[0], dims[1], dims[2], dims[3], p, p, p, p)
        assert L.gpcg_masked_spmv_noalloc(C.byref(st), p, p, p, None, None) == g.ERR_ARG
        assert b"too large" in L.gpcg_last_error()


def test_first_step_mask_box_covers_the_halo():
    """The staged first CG step reads the free bits of columns x0-4 .. x0+67
    (its halo) from one box of 8 mask words whose first word is
    ((x0 >> 5) - 1) rounded down to a multiple of 4: a tensor copy must start
    on a 16-byte boundary, and the box must hold every halo column."""
    for x0 in range(0, 1 << 21, 64):  # chunk columns are multiples of 64
        wx = ((x0 >> 5) - 1) & ~3
        assert wx % 4 == 0
        assert wx <= (x0 - 4) >> 5 and (x0 + 67) >> 5 <= wx + 7


def test_tuner_table_construction():
    """The tuner keys group sizes by tile count: the fastest measured size
    (at least the floor) owns the range up to the geometric mid-point
    towards the next measured size; sizes with equal tile counts are one
    point."""
    from paper_cs_0101018_gb300 import tune
    rows = [(2, 32, 1, {1: 1.0, 2: 2.0, 4: 3.0}, 1),
            (2, 48, 2, {1: 1.0, 2: 0.9, 4: 1.0}, 2),
            (2, 64, 2, {1: 1.0, 2: 0.9, 4: 1.0}, 2),
            (2, 128, 8, {1: 1.0, 2: 2.0, 4: 0.5}, 4),
            (3, 16, 16, {1: 1.0, 2: 2.0, 4: 3.0}, 1)]
    t = tune.table_from(rows)
    assert t[0] == (2, 1, 1, 1) and t[1] == (2, 2, 4, 2) and t[2][:2] == (2, 5)
    assert tune.group_for(t, 2, 3) == 2 and tune.group_for(t, 2, 100) == 4
    assert tune.group_for(t, 3, 10 ** 6) == 1
    t2 = tune.table_from(rows, g_min=2)
    assert tune.group_for(t2, 2, 1) == 2 and tune.group_for(t2, 3, 16) == 2
    assert tune.n_tiles(2, 1600) == 25 * 50 and tune.n_tiles(3, 128) == 2 * 4 * 128
