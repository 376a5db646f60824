"""The five workloads at their full sizes, through the C ABI, in the launch
configuration the benchmark uses.

Where the oracle finishes in seconds (the 1600x1600 QP, small batch members,
reduced 3-D grids) the result is compared with it element by element;
otherwise the properties that hold at any size are checked with the oracle's
own census of the returned point (||grad_Omega q|| <= tau in FP64, x in the box
bit for bit, active/binding counts), plus the agreement of the FP64 and mixed
GPU results within the tolerance implied by the termination test.
Tolerances are those of test_gpu_parity.py."""
import os

import numpy as np
import pytest

import gpcg_inputs as gi
import oracle

g = pytest.importorskip("paper_cs_0101018_gb300")

pytestmark = pytest.mark.gpu


def _rel_err(x, ref):
    return float(np.max(np.abs(x - ref)) / max(1.0, float(np.max(np.abs(ref)))))


def _active_sets_agree(qp, x, ref, band=1e-8):
    act_g = (x == qp.l) | (x == qp.u)
    act_o = (ref == qp.l) | (ref == qp.u)
    near = (np.abs(ref - qp.l) <= band) | (np.abs(ref - qp.u) <= band)
    return bool(np.all((act_g == act_o) | near))


def _check_properties(qp, x, st):
    """Certified at any size: x in Omega exactly and the FP64 census of x (by
    the oracle) meets the tolerance the GPU reported."""
    assert np.all((x >= qp.l) & (x <= qp.u))
    c = oracle.census(qp, x)
    assert np.sqrt(c.pg_norm2) <= st["tau"] * (1 + 1e-9)
    assert c.n_active == st["n_active"]
    assert c.n_binding == st["n_binding"]
    assert np.isclose(c.q, st["q"], rtol=1e-10, atol=1e-10)


@pytest.fixture(scope="module")
def large():
    qp = gi.single_large()
    ref = oracle.solve(qp, tau_rel=1e-8)
    assert ref.status == 0
    return qp, ref


@pytest.mark.parametrize("prec,tol,refine", [(0, 1e-9, 1), (1, 1e-5, 1), (1, 1e-5, 2)])
def test_single_large_matches_oracle(large, prec, tol, refine):
    qp, ref = large
    prob = g.gpcg_problem_create(qp)
    g.gpcg_solve(prob, g.default_options(tau_rel=1e-8, precision=prec, refine=refine))
    x, st = g.gpcg_result(prob)
    assert _rel_err(x, ref.x) <= tol
    assert _active_sets_agree(qp, x, ref.x)
    _check_properties(qp, x, st)


def test_single_large_bench_tolerance_properties():
    """The benchmark's own setting (tau_rel 1e-6, mixed and FP64)."""
    qp = gi.single_large()
    for prec in (g.MIXED, g.FP64):
        prob = g.gpcg_problem_create(qp)
        g.gpcg_solve(prob, g.default_options(tau_rel=1e-6, precision=prec))
        x, st = g.gpcg_result(prob)
        assert st["status"] == 0
        _check_properties(qp, x, st)


def test_precision_stress_3d():
    """128^3 7-point, condition ~1e5: FP64 and mixed (FP32 coefficients with
    the FP64 refinement) both certified by the FP64 census; their distance is
    within what the two termination tests allow (||x - x*|| <= ||pg|| /
    lambda_min for each)."""
    qp = gi.precision_stress()
    res = {}
    for prec in (g.FP64, g.MIXED):
        prob = g.gpcg_problem_create(qp)
        g.gpcg_solve(prob, g.default_options(tau_rel=1e-8, precision=prec))
        x, st = g.gpcg_result(prob)
        assert st["status"] == 0
        _check_properties(qp, x, st)
        res[prec] = (x, st)
    (x64, s64), (x32, s32) = res[g.FP64], res[g.MIXED]
    bound = (s64["pg_norm"] + s32["pg_norm"]) / qp.shift
    assert np.linalg.norm(x64 - x32) <= bound * (1 + 1e-6)
    assert _rel_err(x32, x64) <= 1e-5


GOLDEN_STRESS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden",
                             "precision_stress_128_oracle.npz")


@pytest.fixture(scope="module")
def stress_golden():
    """The oracle's solution of the 128^3 precision-stress QP at tau_rel 1e-12
    (written by tests/golden/make_precision_stress_golden.py: x at 65,536
    seeded sample points, the active set and the 1e-8 band of all points)."""
    d = np.load(GOLDEN_STRESS)
    G = {k: d[k] for k in d.files}
    qp = gi.precision_stress()
    import importlib.util
    spec = importlib.util.spec_from_file_location(
        "make_precision_stress_golden",
        os.path.join(os.path.dirname(GOLDEN_STRESS), "make_precision_stress_golden.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    fp = mk.qp_fingerprint(qp)
    assert mk.fingerprint_matches(fp, G["fingerprint"]), (
        "the generator changed: rewrite the golden file", fp - G["fingerprint"])
    return qp, G


@pytest.mark.parametrize("prec,tol,refine", [(0, 1e-9, 1), (1, 1e-5, 1), (1, 1e-5, 2)])
def test_precision_stress_matches_oracle(stress_golden, prec, tol, refine):
    """The full-size 128^3 anisotropic QP (condition ~1e5) solved to the
    golden's tau_rel: x matches the FP64 oracle at every sampled point within
    the FP64 / mixed tolerance, the active sets agree at every point outside
    the 1e-8 band, and q agrees."""
    qp, G = stress_golden
    prob = g.gpcg_problem_create(qp)
    g.gpcg_solve(prob, g.default_options(tau_rel=float(G["tau_rel"]), precision=prec,
                                         refine=refine))
    x, st = g.gpcg_result(prob)
    assert st["status"] == 0
    idx = G["idx"]
    err = float(np.max(np.abs(x[idx] - G["x_sample"])) / max(1.0, float(G["x_inf"])))
    assert err <= tol, err
    act_o = np.unpackbits(G["active"], count=qp.n).astype(bool)
    near = np.unpackbits(G["near"], count=qp.n).astype(bool)
    act_g = (x == qp.l) | (x == qp.u)
    assert np.all((act_g == act_o) | near)
    assert np.isclose(st["q"], float(G["q"]), rtol=1e-11, atol=0.0)
    _check_properties(qp, x, st)


def test_precision_stress_reduced_matches_oracle():
    """The same generator on a 24^3 grid, where the oracle runs in seconds."""
    qp = gi.precision_stress(24)
    ref = oracle.solve(qp, tau_rel=1e-10)
    for prec, tol in ((g.FP64, 1e-9), (g.MIXED, 1e-5)):
        prob = g.gpcg_problem_create(qp)
        g.gpcg_solve(prob, g.default_options(tau_rel=1e-10, precision=prec))
        x, st = g.gpcg_result(prob)
        assert _rel_err(x, ref.x) <= tol
        assert _active_sets_agree(qp, x, ref.x)


def test_batched_512():
    """512 instances, sides uniform in [64, 512], one engine run (mixed, the
    benchmark's tau_rel 1e-6): every result is certified by the oracle's
    census; a sample is bit-identical to the same instance solved alone
    (oracle parity of batch members at a tight tolerance is the next test)."""
    sides = gi.batch_sides()
    qps = [gi.batch_instance(k, s) for k, s in enumerate(sides)]
    opts = g.default_options(tau_rel=1e-6, precision=g.MIXED)
    probs = [g.gpcg_problem_create(qp) for qp in qps]
    assert g.gpcg_solve_batch(probs, opts, check=False) == 0
    results = [g.gpcg_result(p) for p in probs]
    for qp, (x, st) in zip(qps, results):
        assert st["status"] == 0
        _check_properties(qp, x, st)
    order = np.argsort(sides)
    for k in list(order[:2]) + [int(order[len(order) // 2])]:
        prob = g.gpcg_problem_create(qps[k])
        g.gpcg_solve(prob, opts)
        xa, _ = g.gpcg_result(prob)
        assert np.array_equal(xa, results[k][0])


def _batch_members(count=16):
    """`count` of the 512 batch instances at evenly spaced ranks of their
    sides (64 ... 512), so that both bound kinds and the whole size range
    are represented."""
    sides = gi.batch_sides()
    order = np.argsort(sides, kind="stable")
    ks = [int(order[int(round(j * (len(order) - 1) / (count - 1)))]) for j in range(count)]
    return [gi.batch_instance(k, sides[k]) for k in ks]


@pytest.fixture(scope="module")
def batch_members():
    qps = _batch_members()
    kinds = {"lower0" if np.all(np.isinf(q.u)) else "two_sided" for q in qps}
    assert kinds == {"lower0", "two_sided"}
    oracle.set_threads(0)
    refs = [oracle.solve(qp, tau_rel=1e-10) for qp in qps]
    oracle.set_threads(1)
    assert all(r.status == 0 for r in refs)
    return qps, refs


@pytest.mark.parametrize("prec,tol,refine", [(0, 1e-9, 1), (1, 1e-5, 1), (1, 1e-5, 2)])
def test_batched_members_match_oracle(batch_members, prec, tol, refine):
    """Sixteen of the 512 batched instances (sides 64 ... 512, one- and
    two-sided bounds) solved in one batch at tau_rel 1e-10: every member
    matches the oracle element by element within the FP64 / mixed tolerance,
    with identical active sets outside the 1e-8 band."""
    qps, refs = batch_members
    probs = [g.gpcg_problem_create(qp) for qp in qps]
    opts = g.default_options(tau_rel=1e-10, precision=prec, refine=refine)
    assert g.gpcg_solve_batch(probs, opts, check=False) == 0
    for qp, ref, prob in zip(qps, refs, probs):
        x, st = g.gpcg_result(prob)
        assert st["status"] == 0
        assert _rel_err(x, ref.x) <= tol, (qp.name, _rel_err(x, ref.x))
        assert _active_sets_agree(qp, x, ref.x), qp.name
        _check_properties(qp, x, st)


# The server runs every request on the pass engine, so the solo solves its
# results are compared with bit for bit take the engine too (path=ENGINE); a
# small QP alone would otherwise go to the resident solver.


def _served(qps, opts, max_live=4):
    srv = g.Server(hbm_budget=2 << 30, max_live=max_live, opts=opts)
    tickets = []
    pending = list(qps)
    while pending or any(not srv.done(t) for t in tickets):
        for _ in range(2):
            if pending:
                tickets.append(srv.submit(pending.pop(0)))
        srv.step(16)
    out = []
    for tk in tickets:
        st, _ = srv.stats(tk)
        out.append((tk.x, st))
    srv.close()
    return out


@pytest.mark.parametrize("prec,tol", [(0, 1e-9), (1, 1e-5)])
def test_served_results_match_oracle(prec, tol):
    """Requests of the serving trace (2-D and 3-D, all three bound kinds),
    served with continuous batching at tau_rel 1e-10: each served x matches
    the oracle within the FP64 / mixed tolerance (active sets outside the
    1e-8 band identical) and is bit-identical to the same QP solved alone."""
    reqs = [r for r in gi.serving_trace(rate=200.0, duration=3.0) if
            (r.side ** r.dim) <= 120_000][:12]
    assert any(r.dim == 3 for r in reqs) and any(r.dim == 2 for r in reqs)
    assert len({r.bounds for r in reqs}) == 3
    qps = [gi.serving_instance(r) for r in reqs]
    opts = g.default_options(path=g.PATH_ENGINE, tau_rel=1e-10, precision=prec)
    served = _served(qps, opts)
    oracle.set_threads(0)
    try:
        for qp, (x, st) in zip(qps, served):
            assert st["status"] == 0
            ref = oracle.solve(qp, tau_rel=1e-10)
            assert ref.status == 0
            assert _rel_err(x, ref.x) <= tol, (qp.name, _rel_err(x, ref.x))
            assert _active_sets_agree(qp, x, ref.x), qp.name
            prob = g.gpcg_problem_create(qp)
            g.gpcg_solve(prob, opts)
            xa, _ = g.gpcg_result(prob)
            assert np.array_equal(xa, x), qp.name
    finally:
        oracle.set_threads(1)


def test_serving_same_alone_and_in_the_mix():
    """Continuous batching: requests of different sizes and dimensions arrive
    while others run; each result equals the same QP solved alone, bit for
    bit, and latencies are recorded."""
    reqs = [r for r in gi.serving_trace(rate=200.0, duration=2.0) if
            (r.side ** r.dim) <= 300_000][:24]
    assert len(reqs) >= 12 and any(r.dim == 3 for r in reqs)
    qps = [gi.serving_instance(r) for r in reqs]
    opts = g.default_options(path=g.PATH_ENGINE, tau_rel=1e-6, precision=g.MIXED)
    srv = g.Server(hbm_budget=2 << 30, max_live=8, opts=opts)
    tickets = []
    pending = list(qps)
    # submit in waves so that new requests join while earlier ones are live
    while pending or any(not srv.done(t) for t in tickets):
        for _ in range(3):
            if pending:
                tickets.append(srv.submit(pending.pop(0)))
        srv.step(16)
    lat = []
    for qp, tk in zip(qps, tickets):
        st, latency = srv.stats(tk)
        assert st["status"] == 0
        lat.append(latency)
        prob = g.gpcg_problem_create(qp)
        g.gpcg_solve(prob, opts)
        xa, _ = g.gpcg_result(prob)
        assert np.array_equal(xa, tk.x)
    q, r, f = srv.counts()
    assert (q, r, f) == (0, 0, len(qps))
    assert all(l > 0 for l in lat)
    t = srv.timing()
    assert t["steps"] >= t["steps_with_passes"] > 0 and t["device_passes"] > 0
    assert min(t.values()) >= 0.0
    srv.close()


def test_serving_budget_and_cancel():
    qp_big = gi.grid_qp_2d(400, 400, seed=9, shift=1e-2)
    qp_small = gi.grid_qp_2d(50, 50, seed=10, shift=1e-2)
    opts = g.default_options(path=g.PATH_ENGINE, tau_rel=1e-6, precision=g.FP64)
    srv = g.Server(hbm_budget=8 << 20, max_live=4, opts=opts)
    with pytest.raises(g.GpcgError) as e:
        srv.submit(qp_big)  # 160k points do not fit an 8 MB budget at all
    assert e.value.status == g.ERR_BUDGET
    t1 = srv.submit(qp_small)
    t2 = srv.submit(qp_small)
    srv.cancel(t2)
    while not srv.done(t1):
        srv.step(16)
    st, _ = srv.stats(t1)
    assert st["status"] == 0
    with pytest.raises(g.GpcgError) as e:
        srv.stats(t2)
    assert e.value.status == g.ERR_CANCELLED
    srv.close()


@pytest.mark.parametrize("opt", [dict(precond=1), dict(precond=2), dict(cg_system=1),
                                 dict(precision=0)])
def test_serving_with_options_same_alone_and_in_the_mix(opt):
    """The server runs the options' own pass kernel (point Jacobi, the tile
    preconditioner, the explicit reduced system, FP64): each result equals the
    same QP solved alone, bit for bit."""
    qps = [gi.grid_qp_2d(nx, ny, seed=600 + k, shift=1e-2, bounds="two_sided")
           for k, (nx, ny) in enumerate([(200, 150), (64, 64), (300, 90), (130, 70), (70, 300)])]
    base = dict(tau_rel=1e-6, precision=g.MIXED, path=g.PATH_ENGINE)
    base.update(opt)
    opts = g.default_options(**base)
    srv = g.Server(hbm_budget=1 << 30, max_live=3, opts=opts)
    tickets = [srv.submit(qp) for qp in qps]
    while any(not srv.done(t) for t in tickets):
        srv.step(16)
    for qp, tk in zip(qps, tickets):
        st, _ = srv.stats(tk)
        assert st["status"] == 0
        prob = g.gpcg_problem_create(qp)
        g.gpcg_solve(prob, opts)
        xa, _ = g.gpcg_result(prob)
        assert np.array_equal(xa, tk.x)
    srv.close()


def test_serving_input_checks_in_the_mix():
    """A request's input checks run on the device when it takes its slot: an
    empty box or a NaN in b ends that request with its error status, and the
    requests served in the same steps match their solo solves bit for bit."""
    import dataclasses
    good = [gi.grid_qp_2d(60 + 7 * k, 50, seed=700 + k, shift=1e-2, bounds="two_sided")
            for k in range(3)]
    base = gi.grid_qp_2d(40, 40, seed=710, shift=1e-2, bounds="two_sided")
    l_bad = base.l.copy()
    l_bad[5] = base.u[5] + 0.25
    empty_box = dataclasses.replace(base, l=l_bad)
    b_bad = base.b.copy()
    b_bad[7] = np.nan
    nan_b = dataclasses.replace(base, b=b_bad)
    qps = [good[0], empty_box, good[1], nan_b, good[2]]
    opts = g.default_options(path=g.PATH_ENGINE, tau_rel=1e-6, precision=g.MIXED)
    srv = g.Server(hbm_budget=1 << 30, max_live=4, opts=opts)
    tickets = [srv.submit(qp) for qp in qps]
    while any(not srv.done(t) for t in tickets):
        srv.step(16)
    status = [srv.stats(t)[0]["status"] for t in tickets]
    assert status == [0, g.ERR_INFEASIBLE, 0, g.ERR_ARG, 0]
    for qp, tk in ((good[0], tickets[0]), (good[1], tickets[2]), (good[2], tickets[4])):
        prob = g.gpcg_problem_create(qp)
        g.gpcg_solve(prob, opts)
        xa, _ = g.gpcg_result(prob)
        assert np.array_equal(xa, tk.x)
    assert srv.counts() == (0, 0, len(qps))
    srv.close()


def test_serving_pinned_and_pageable_buffers_give_the_same_result():
    """Requests in pinned host memory are copied by DMA directly, ordinary
    (pageable) ones through the workers' staging buffers; results go to a
    caller-given x_out or to a new array.  Both routes give the same x."""
    import dataclasses
    import torch
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    qps = [gi.grid_qp_2d(97, 61, seed=720, shift=1e-2, bounds="two_sided"),
           gi.grid_qp_3d(13, 11, 9, seed=721, shift=1e-2, sigma=0.5, bounds="lower0",
                         b_dist="uniform")]
    opts = g.default_options(path=g.PATH_ENGINE, tau_rel=1e-6, precision=g.MIXED)
    srv = g.Server(hbm_budget=1 << 30, max_live=4, opts=opts)
    plain = [srv.submit(q) for q in qps]
    pinned_qps = [dataclasses.replace(q, diag=pin(q.diag), cx=pin(q.cx), cy=pin(q.cy),
                                      cz=pin(q.cz) if q.cz is not None else None,
                                      b=pin(q.b), l=pin(q.l), u=pin(q.u)) for q in qps]
    outs = [pin(np.zeros(q.n)) for q in qps]
    pinned = [srv.submit(q, x_out=o) for q, o in zip(pinned_qps, outs)]
    while any(not srv.done(t) for t in plain + pinned):
        srv.step(16)
    for a, b, o in zip(plain, pinned, outs):
        assert srv.stats(a)[0]["status"] == 0 and srv.stats(b)[0]["status"] == 0
        assert b.x is o
        assert np.array_equal(a.x, b.x)
    srv.close()


def test_serving_cancel_in_any_state_and_close_with_work_in_flight():
    """Cancelling requests wherever they are (queued, uploading, running or
    being read back) ends them cancelled and leaves the others exact; a
    server closed with requests in flight shuts down cleanly."""
    qps = [gi.grid_qp_2d(40 + 9 * k, 30 + 5 * k, seed=730 + k, shift=1e-2, bounds="two_sided")
           for k in range(10)]
    opts = g.default_options(path=g.PATH_ENGINE, tau_rel=1e-6, precision=g.MIXED)
    srv = g.Server(hbm_budget=1 << 30, max_live=3, opts=opts)
    tickets = [srv.submit(q) for q in qps]
    cancelled = set()
    for step in range(6):
        srv.step(4)
        k = 1 + 3 * step
        if k < len(tickets):
            try:
                srv.cancel(tickets[k])
                cancelled.add(k)
            except g.GpcgError as e:
                # a worker finished it first
                assert e.status == g.ERR_ARG and srv.done(tickets[k])
    while True:
        q, r, f = srv.counts()
        if q + r == 0:
            break
        srv.step(16)
    assert f == len(qps)
    for k, (qp, tk) in enumerate(zip(qps, tickets)):
        if k in cancelled:
            with pytest.raises(g.GpcgError) as e:
                srv.stats(tk)
            assert e.value.status == g.ERR_CANCELLED
            continue
        st, _ = srv.stats(tk)
        assert st["status"] == 0
        prob = g.gpcg_problem_create(qp)
        g.gpcg_solve(prob, opts)
        xa, _ = g.gpcg_result(prob)
        assert np.array_equal(xa, tk.x)
    srv.close()
    # closed while requests are queued, uploading and running
    srv = g.Server(hbm_budget=1 << 30, max_live=2, opts=opts)
    for q in qps:
        srv.submit(q)
    srv.step(4)
    srv.step(4)
    srv.close()
