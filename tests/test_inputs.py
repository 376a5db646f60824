"""CPU checks of the seeded workload generators that the serving benchmark
relies on (no solver arithmetic here)."""
import math

import numpy as np

import gpcg_inputs as gi


def test_serving_trace_is_seeded_and_a_prefix_of_the_full_trace():
    short = gi.serving_trace(duration=2.0)
    full = gi.serving_trace(duration=6.0)
    assert short == full[:len(short)]
    assert all(a.t_arrival < b.t_arrival for a, b in zip(full, full[1:]))
    assert gi.serving_trace(duration=2.0) == short
    # Poisson at 200/s: about 400 arrivals in 2 s
    assert 300 < len(short) < 500


def test_serving_pool_sides_span_the_size_range():
    for dim in (2, 3):
        sides = gi.serving_pool_sides(dim)
        assert np.all(np.diff(sides) > 0)
        n = sides.astype(float) ** dim
        assert n[0] <= 1.5e3 and n[-1] >= 3.5e6
        # log-spaced: consecutive sizes differ by a bounded ratio
        assert np.max(n[1:] / n[:-1]) < 1.8


def test_pool_side_is_nearest_in_log_n():
    sides = {d: gi.serving_pool_sides(d) for d in (2, 3)}
    for r in gi.serving_trace(duration=1.0):
        s = gi.pool_side(r, sides[r.dim])
        best = min(sides[r.dim], key=lambda c: abs(math.log(c) - math.log(r.side)))
        assert s == best


def test_with_bounds_shares_the_hessian_and_sets_the_kind():
    qp = gi.grid_qp_2d(12, 9, seed=3, shift=1e-2, bounds="box1")
    lo = gi.with_bounds(qp, "lower0", 3)
    ts = gi.with_bounds(qp, "two_sided", 3)
    for q in (lo, ts):
        assert q.diag is qp.diag and q.cx is qp.cx and q.b is qp.b
    assert np.all(lo.l == 0.0) and np.all(np.isinf(lo.u))
    assert np.all((ts.l >= -0.5) & (ts.l <= 0.0)) and np.all((ts.u >= 0.0) & (ts.u <= 0.5))
    assert np.all(qp.l == -1.0) and np.all(qp.u == 1.0)


def test_serving_pool_covers_every_dimension_size_and_bound_kind():
    pool = gi.serving_pool(count=4)
    for dim in (2, 3):
        for side in gi.serving_pool_sides(dim, 4):
            for kind in ("lower0", "two_sided", "box1"):
                q = pool[(dim, int(side), kind)]
                assert q.dim == dim and q.nx == side and q.n == side ** dim


def test_disc_free_qp_is_free_on_its_disc():
    """The free-set ablation workload: the oracle's solution is free on the
    whole disc and at its bound beyond a thin band around it (a few cells, the
    reach of the Laplacian's coupling), so the free fraction follows the disc."""
    import oracle
    side = 64
    fracs = []
    for frac in (0.1, 0.3, 0.6):
        qp = gi.disc_free_qp(side, frac)
        r = oracle.solve(qp, tau_rel=1e-10)
        assert r.status == oracle.OK
        iy, ix = np.divmod(np.arange(side * side), side)
        c = (side - 1) / 2.0
        d = np.hypot(ix - c, iy - c) - side * math.sqrt(frac / math.pi)
        free = r.x > 0.0
        assert np.all(free[d <= 0.0])
        assert np.max(d[free]) <= 8.0
        fracs.append(float(np.mean(free)))
    assert fracs[0] < fracs[1] < fracs[2]


def test_precision_stress_golden_is_current():
    """The stored oracle solution of the 128^3 precision-stress QP belongs to
    the current generator (same fingerprint of the arrays, same sample points),
    lies in the box, and meets its own termination test."""
    import importlib.util
    import os
    here = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    spec = importlib.util.spec_from_file_location(
        "make_precision_stress_golden", os.path.join(here, "make_precision_stress_golden.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    d = np.load(mk.OUT)
    qp = gi.precision_stress()
    assert mk.fingerprint_matches(mk.qp_fingerprint(qp), d["fingerprint"])
    assert int(d["n"]) == qp.n
    assert np.array_equal(d["idx"], mk.sample_indices(qp.n))
    xs = d["x_sample"]
    assert np.all((xs >= qp.l[d["idx"]]) & (xs <= qp.u[d["idx"]]))
    assert float(d["x_inf"]) >= float(np.max(np.abs(xs)))
    assert float(d["pg_norm"]) <= float(d["tau_rel"]) * float(d["pg_norm0"])
    act = np.unpackbits(d["active"], count=qp.n).astype(bool)
    near = np.unpackbits(d["near"], count=qp.n).astype(bool)
    assert np.all(near[act])  # a point at a bound is within the band
    assert int(d["stats"][4]) == int(act.sum())
