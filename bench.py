#!/usr/bin/env python
"""Benchmark: GPCG solves/s on the single large QP (2-D 1600x1600, n = 2.56e6,
5-point weighted-Laplacian Hessian with shift 1e-3, b ~ U[-1,1], two-sided
bounds l ~ U[-0.5,0], u ~ U[0,0.5], seed 2), stopping at
||grad_Omega q(x)|| <= 1e-6 ||grad_Omega q(x0)||.

One step = one complete GPCG solve (every pass of the hot path) of that QP.
`value` is the mixed-precision (FP32-stream / FP64-reduce) rate; the plain
FP64 path is reported beside it.  Inputs are resident in HBM before the
timed region; `e2e` repeats the measurement through the C ABI with pinned
host buffers (each step: the QP's copies in, overlapped with the previous
step's solve, the solve, and the read-back of x).  The same line reports the
masked product alone, the preconditioners, the journal bearing, the
extracted reduced system, the 32x32 and 128^3 QPs, the 512-QP batch and the
serving trace (`--serve-seconds`, 0 to skip the last two).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank solves its own replica (weak scaling, no collective
in the data path; a barrier brackets the timed region).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gpcg_inputs as gi  # noqa: E402

WORKLOAD = "single_large_2d_1600x1600"
METRIC = "GPCG solves/s (single large QP, 1600x1600 5-point, tau_rel 1e-6)"
TAU_REL = 1e-6


TRAFFIC_FILE = os.path.join(ROOT, "profiles", "pass_kernel_traffic_single_large_1600.json")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_cs_0101018_gb300", "csrc", f)
                  for f in ("pass_engine.cuh", "gpcg_kernels.cu", "engine.h", "gpcg_coop.cu",
                            "gpcg_coop_f64.cu")]


def _kernel_sha():
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def _traffic():
    """DRAM bytes per pass of the benchmark solve, from the committed ncu
    summary (JSON), or None when the kernel sources changed since it was
    taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            kv = json.load(f)
        if kv.get("kernel_sources_sha256") != _kernel_sha():
            return None, None
        return float(kv["mixed_dram_bytes_per_pass"]), float(kv["fp64_dram_bytes_per_pass"])
    except Exception:
        return None, None


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.file, stderr=subprocess.DEVNULL)
            # the timed region starts once the sampler runs (first row written)
            t0 = time.perf_counter()
            while time.perf_counter() - t0 < 3.0 and self.proc.poll() is None:
                if os.path.getsize(self.file.name) > 0:
                    break
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.file:
            return None
        try:
            with open(self.file.name) as f:
                rows = [r.split(",") for r in f.read().strip().splitlines() if r.strip()]
            os.unlink(self.file.name)
        except Exception:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    import torch.distributed as dist
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1 and not dist.is_initialized():
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return ws, int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def _max_over_ranks(ws, v):
    if ws == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available()
                     else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def host_cpu():
    """The host's processor count and model (from os and /proc/cpuinfo or
    lscpu), recorded beside the oracle's timings."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() in ("Model name", "Model"):
                if model is None or k.strip() == "Model name":
                    model = v.strip()
    except Exception:
        pass
    return {"nproc": os.cpu_count(), "model": model}


def _oracle_solves(qp, threads: int, budget_s: float, max_solves: int):
    """Complete oracle solves on `threads` row-loop threads until about
    budget_s seconds have passed (at least one); returns (solves/s, solves,
    threads in force, status)."""
    import oracle
    used = oracle.set_threads(threads)
    try:
        t0 = time.perf_counter()
        k = 0
        while True:
            r = oracle.solve(qp, tau_rel=TAU_REL)
            k += 1
            if time.perf_counter() - t0 > budget_s or k >= max_solves:
                break
        return k / (time.perf_counter() - t0), k, used, r.status
    finally:
        oracle.set_threads(1)


def cpu_baseline(qp, budget_s: float = 25.0):
    """The oracle as it stands, timed on the host: on one core, and with its
    row loops (matrix-vector products, projections, vector updates) on every
    core (its sums stay sequential, so both give the same x bit for bit).
    `value` is the all-core figure; about budget_s seconds in all."""
    import oracle
    v1, k1, _, s1 = _oracle_solves(qp, 1, budget_s * 0.5, 3)
    va, ka, used, sa = _oracle_solves(qp, 0, budget_s * 0.5, 6)
    # the 32x32 QP (tau_rel 1e-8) on one core: its latency beside the GPU's
    sq = gi.single_small()
    oracle.solve(sq, tau_rel=1e-8)
    ms = []
    for _ in range(50):
        t0 = time.perf_counter()
        oracle.solve(sq, tau_rel=1e-8)
        ms.append(1000.0 * (time.perf_counter() - t0))
    ms.sort()
    return {"value": va, "unit": "solves/s", "cores": used, "kind": "oracle",
            "sample": f"{ka} complete FP64 solve(s) of the 1600x1600 workload with the row "
                      f"loops on {used} threads; {k1} on one core",
            "single_core": {"value": v1, "unit": "solves/s", "cores": 1, "solves": k1},
            "single_small_32": {"p50_ms": ms[len(ms) // 2], "p99_ms": ms[-1], "cores": 1,
                                "solves": len(ms)},
            "host": host_cpu(), "status": max(s1, sa)}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    qp = gi.single_large()
    import oracle
    oracle.build()
    used = oracle.set_threads(0)
    times = []
    for _ in range(args.warmup):
        oracle.solve(qp, tau_rel=TAU_REL)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.solve(qp, tau_rel=TAU_REL)
        times.append(time.perf_counter() - t0)
    oracle.set_threads(1)
    tot = sum(times)
    value = args.steps / tot
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * tot / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": qp.n, "tau_rel": TAU_REL},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": used, "kind": "oracle",
                             "sample": "one complete FP64 solve of the 1600x1600 workload "
                                       f"per step, row loops on {used} threads",
                             "host": host_cpu()},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "status": r.status}
    print(json.dumps(line), flush=True)


def bench_batched(g, stream, reps: int = 2) -> dict:
    """The batched workload: 512 2-D QPs with sides uniform on {64..512}, all
    advanced by one engine run (`gpcg_solve_batch`), mixed and FP64."""
    import torch
    sides = gi.batch_sides()
    qps = [gi.batch_instance(k, s) for k, s in enumerate(sides)]
    probs = [g.gpcg_problem_create(qp) for qp in qps]
    out = {"instances": len(qps), "unknowns": int(sum(q.n for q in qps))}
    del qps
    for name, prec in (("mixed", g.MIXED), ("fp64", g.FP64)):
        opts = g.default_options(tau_rel=TAU_REL, precision=prec, stream=stream)
        g.gpcg_solve_batch(probs, opts)
        ms = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.gpcg_solve_batch(probs, opts)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        sts = [g.gpcg_result(p, None)[1] for p in probs]
        t = min(ms)
        out[name] = {"solves/s": len(probs) / (t / 1000.0), "ms_per_batch": t,
                     "passes": int(max(st["passes"] for st in sts)),
                     "cg_iters_total": int(sum(st["cg_iters"] for st in sts)),
                     "all_converged": all(st["status"] == 0 for st in sts)}
    del probs
    return out


def serve_trace(g, pool, reqs, opts, realtime: bool, max_live: int = 128,
                passes: int = 16) -> dict:
    """Replays a request trace through the continuous-batching server.

    realtime: each request is submitted at its arrival time (latency = server
    latency + the wait for the host loop); otherwise requests are submitted
    as fast as the server takes them, keeping 2 * max_live outstanding, and
    the figure is the server's capacity (requests / makespan)."""
    sides = {d: gi.serving_pool_sides(d) for d in (2, 3)}
    srv = g.Server(hbm_budget=150 << 30, max_live=max_live, opts=opts)
    lat = [0.0] * len(reqs)
    pend = {}
    i = finished = bad = steps = 0
    last_counts, t_change = None, time.perf_counter()
    t0 = time.perf_counter()
    while True:
        now = time.perf_counter() - t0
        while i < len(reqs) and (reqs[i].t_arrival <= now if realtime
                                  else i - finished < 2 * max_live):
            r = reqs[i]
            tk = srv.submit(pool[(r.dim, gi.pool_side(r, sides[r.dim]), r.bounds)])
            pend[tk.id] = (i, tk, r.t_arrival if realtime else 0.0, time.perf_counter() - t0)
            i += 1
        # one consistent snapshot: results are read back by the server's
        # workers, so requests also finish between steps
        q, run, f = srv.counts()
        if (q, run, f) != last_counts:
            last_counts, t_change = (q, run, f), time.perf_counter()
        elif time.perf_counter() - t_change > 120.0:
            raise RuntimeError(f"server made no progress for 120 s: queued {q}, running {run}, "
                               f"finished {f} of {len(reqs)}")
        if f > finished:
            for tid in [t for t, v in pend.items() if srv.done(v[1])]:
                k, tk, ta, ts = pend.pop(tid)
                st, l = srv.stats(tk)
                lat[k] = l + (ts - ta)
                bad += st["status"] != 0
                srv.release(tk)
            finished = f
        if finished >= len(reqs):
            break
        if q + run == 0:
            if realtime and i < len(reqs):
                time.sleep(max(0.0, reqs[i].t_arrival - (time.perf_counter() - t0)))
            continue
        srv.step(passes)
        steps += 1
    wall = time.perf_counter() - t0
    timing = {k: round(v, 4) for k, v in srv.timing().items()}
    srv.close()
    lat.sort()
    pq = lambda q: 1000.0 * lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
    return {"solves/s": len(reqs) / wall, "wall_s": wall, "p50_ms": pq(0.5), "p99_ms": pq(0.99),
            "max_ms": 1000.0 * lat[-1], "server_steps": steps, "failed": bad,
            "server_timing_s": timing}


def bench_serving(g, seconds: float) -> dict:
    """The serving workload: Poisson arrivals at 200/s, n log-uniform on
    [1e3, 4e6], 70 % 2-D / 30 % 3-D, three bound kinds, 150 GB budget; mixed
    and FP64, replayed in real time and queued at once (capacity)."""
    # requests arrive in ordinary (pageable) numpy arrays and their results
    # go to new ones; the server's workers stage both through pinned buffers
    pool = gi.serving_pool()
    reqs = gi.serving_trace(duration=seconds)
    sides = {d: gi.serving_pool_sides(d) for d in (2, 3)}
    out = {"trace_s": seconds, "requests": len(reqs),
           "unknowns_trace": int(sum(r.side ** r.dim for r in reqs)),
           "unknowns_served": int(sum(gi.pool_side(r, sides[r.dim]) ** r.dim for r in reqs)),
           "pool": "24 log-spaced sizes per dimension x 3 bound kinds; a request takes "
                   "the pool QP of its dimension and bound kind nearest in log n",
           "max_live": 128, "hbm_budget_GB": 150,
           "host_buffers": "numpy arrays (pageable), inputs and results"}
    for name, prec in (("mixed", g.MIXED), ("fp64", g.FP64)):
        opts = g.default_options(tau_rel=TAU_REL, precision=prec)
        serve_trace(g, pool, reqs[:64], opts, realtime=False)  # warm-up
        out[name] = {"realtime": serve_trace(g, pool, reqs, opts, realtime=True),
                     "capacity": serve_trace(g, pool, reqs, opts, realtime=False)}
    out["mixed_over_fp64_capacity"] = (out["mixed"]["capacity"]["solves/s"] /
                                       out["fp64"]["capacity"]["solves/s"])
    return out


def run_ours(args):
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    import paper_cs_0101018_gb300 as g
    g.load()
    qp = gi.single_large()
    stream = torch.cuda.Stream()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    d_in = {k: dev(getattr(qp, k)) for k in ("diag", "cx", "cy", "b", "l", "u")}
    torch.cuda.synchronize()
    prob = g.gpcg_problem_create(dim=2, nx=qp.nx, ny=qp.ny, **d_in)
    hbm_peak, peak_kind = _peaks()

    def timed(precision, steps, warmup, precond=0, refine=2):
        opts = g.default_options(tau_rel=TAU_REL, precision=precision, stream=stream,
                                 precond=precond, refine=refine)
        for _ in range(warmup):
            g.gpcg_solve(prob, opts)
        torch.cuda.synchronize()
        _barrier(ws)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        with Clocks(local) as clk:
            t_wall = time.perf_counter()
            for e0, e1 in ev:
                e0.record(stream)
                g.gpcg_solve(prob, opts)
                e1.record(stream)
                e1.synchronize()
            torch.cuda.synchronize()
            t_wall = time.perf_counter() - t_wall
        _barrier(ws)
        torch.cuda.synchronize()
        ms = [a.elapsed_time(b) for a, b in ev]
        _, st = g.gpcg_result(prob)
        return ms, st, clk.summary(), t_wall

    # mixed precision (headline) and plain FP64
    ms_mx, st_mx, clk_mx, wall_mx = timed(g.MIXED, args.steps, args.warmup)
    ms_64, st_64, clk_64, wall_64 = timed(g.FP64, args.steps, args.warmup)
    # mixed with the FP64 phase's CG phases in FP64 (refine 1; the default,
    # refine 2, runs them as FP32 correction solves on the FP64 gradient)
    ms_r1, st_r1, _, _ = timed(g.MIXED, max(1, min(args.steps, 20)), 2, refine=1)
    # the preconditioned CG phases (Sec. 6) on the same workload: point
    # Jacobi and the tile block Jacobi (zebra line sweep in 64 x 8 tiles)
    jac, tile = {}, {}
    for out, pc in ((jac, g.PRECOND_JACOBI), (tile, g.PRECOND_TILE)):
        for name, prec in (("mixed", g.MIXED), ("fp64", g.FP64)):
            msj, stj, _, _ = timed(prec, max(1, min(args.steps, 5)), 1, precond=pc)
            tj = _max_over_ranks(ws, sum(msj) / 1000.0)
            out[name] = {"value": ws * len(msj) / tj, "unit": "solves/s",
                         "ms_per_step": sum(msj) / len(msj),
                         "solve": {k: stj[k] for k in ("outer_iters", "gp_iters", "cg_iters",
                                                       "passes", "pg_norm", "tau")}}

    tot_mx = _max_over_ranks(ws, sum(ms_mx) / 1000.0)
    tot_64 = _max_over_ranks(ws, sum(ms_64) / 1000.0)
    value = ws * args.steps / tot_mx
    value_64 = ws * args.steps / tot_64

    traffic_mx, traffic_64 = _traffic()

    def roof(ms, st, traffic):
        # per pass of the solve: algorithmic bytes / (solve time / passes); the
        # solve time includes the gaps between passes, so this is conservative
        t = (sum(ms) / len(ms)) / 1000.0
        per_pass_t = t / max(1, st["passes"])
        per_pass_b = st["alg_bytes"] / max(1, st["passes"])
        ach = per_pass_b / per_pass_t / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                "frac": ach / hbm_peak, "traffic": traffic, "peak_kind": peak_kind,
                "kernel": "gpcg::pass_kernel", "alg_bytes_per_launch": per_pass_b,
                "launch_ms": 1000 * per_pass_t,
                "note": "per engine pass of one solve (all passes of a lone solve run in one "
                        "cooperative launch); time = solve time / passes"}

    roof_mx, roof_64 = roof(ms_mx, st_mx, traffic_mx), roof(ms_64, st_64, traffic_64)

    # masked product alone (y = Z Z' A Z Z' p and <p, y>, B = n (k_c s + 2 s) +
    # n/8 bytes), on the solve's final free set, then on a 4096^2 grid of the
    # same generator where a single launch is no longer dominated by its fixed
    # costs (launch, first copies, final reduction)
    spmv = {}
    for name, prec in (("mixed", g.MIXED), ("fp64", g.FP64)):
        g.gpcg_solve(prob, g.default_options(tau_rel=TAU_REL, precision=prec, stream=stream))
        ms1, by = g.gpcg_time_masked_spmv(prob, prec, reps=20, flush_l2=True, stream=stream)
        ms2, _ = g.gpcg_time_masked_spmv(prob, prec, reps=20, flush_l2=False, stream=stream)
        gbs = by / (ms1 / 1000.0) / 1e9
        spmv[name] = {"GB/s": gbs, "frac": gbs / hbm_peak, "ms_per_launch": ms1,
                      "alg_bytes_per_launch": by, "grid": [qp.nx, qp.ny],
                      "l2": "flushed before each launch",
                      "GB/s_l2_warm": by / (ms2 / 1000.0) / 1e9,
                      "kernel": "gpcg::mspmv_kernel"}
    # the same kernel as an iterative method issues it: back-to-back launches
    # over 6 distinct 1600^2 problems of the generator (seeds 2, 11..15;
    # their operands, 6 x 51 MB mixed and 6 x 103 MB FP64, exceed the L2
    # twice over, so each launch streams from HBM), each launch free to start
    # while the previous one drains
    sprobs = [prob] + [g.gpcg_problem_create(gi.grid_qp_2d(qp.nx, qp.ny, seed=sd, shift=1e-3,
                                                           bounds="two_sided"))
                       for sd in (11, 12, 13, 14, 15)]
    for name, prec in (("mixed_stream", g.MIXED), ("fp64_stream", g.FP64)):
        for sp_ in sprobs:
            g.gpcg_solve(sp_, g.default_options(tau_rel=TAU_REL, precision=prec, stream=stream))
        ms1, by = g.gpcg_time_masked_spmv_stream(sprobs, prec, reps=10, stream=stream)
        gbs = by / (ms1 / 1000.0) / 1e9
        spmv[name] = {"GB/s": gbs, "frac": gbs / hbm_peak, "ms_per_launch": ms1,
                      "alg_bytes_per_launch": by, "grid": [qp.nx, qp.ny],
                      "l2": "6 distinct problems in turn (operands > 2x L2)",
                      "launches": 10 * len(sprobs), "kernel": "gpcg::mspmv_kernel"}
    del sprobs
    big = gi.grid_qp_2d(4096, 4096, seed=2, shift=1e-3, bounds="two_sided")
    pbig = g.gpcg_problem_create(big)
    for name, prec in (("mixed_4096", g.MIXED), ("fp64_4096", g.FP64)):
        ms1, by = g.gpcg_time_masked_spmv(pbig, prec, reps=20, flush_l2=True, stream=stream)
        gbs = by / (ms1 / 1000.0) / 1e9
        spmv[name] = {"GB/s": gbs, "frac": gbs / hbm_peak, "ms_per_launch": ms1,
                      "alg_bytes_per_launch": by, "grid": [big.nx, big.ny],
                      "l2": "flushed before each launch (inputs > L2)",
                      "kernel": "gpcg::mspmv_kernel"}
    del pbig, big

    # the journal bearing problem of Sec. 5 (finite differences, 1600^2 like
    # the paper's n = 2.56e6; tau = 1e-4 absolute, x0 = l), with the point-
    # Jacobi and the tile preconditioned CG phases
    jb = {}
    for eps in (0.1, 0.9):
        jqp = gi.journal_bearing(1600, 1600, eps)
        jp = g.gpcg_problem_create(jqp)
        for name, prec, pc in (("mixed_jacobi", g.MIXED, g.PRECOND_JACOBI),
                               ("mixed_tile", g.MIXED, g.PRECOND_TILE),
                               ("fp64_jacobi", g.FP64, g.PRECOND_JACOBI),
                               ("fp64_tile", g.FP64, g.PRECOND_TILE)):
            jo = g.default_options(tau_abs=1e-4, tau_rel=0.0, precision=prec, precond=pc,
                                   stream=stream)
            g.gpcg_solve(jp, jo)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.gpcg_solve(jp, jo)
            e1.record(stream)
            e1.synchronize()
            xj, sj = g.gpcg_result(jp)
            jb[f"eps{eps}_{name}"] = {
                "solves/s": 1000.0 / e0.elapsed_time(e1), "ms": e0.elapsed_time(e1),
                "outer_iters": sj["outer_iters"], "gp_iters": sj["gp_iters"],
                "cg_iters": sj["cg_iters"], "free_fraction": float(np.mean(xj > 0)),
                "pg_norm": sj["pg_norm"], "status": sj["status"]}
        del jp, jqp

    # the reduced system applied through the bitmask (the default) or
    # extracted into compact numbering (Sec. 4's A_k), on 1600^2 QPs whose
    # solutions are free on a disc covering the given fraction of the grid
    ablation = {}
    for frac in (0.01, 0.1, 0.3, 0.9):
        dqp = gi.disc_free_qp(1600, frac)
        dp = g.gpcg_problem_create(dqp)
        row = {}
        for name, cs in (("masked", g.CG_MASKED), ("extracted", g.CG_EXTRACTED)):
            do = g.default_options(tau_rel=TAU_REL, precision=g.MIXED, cg_system=cs,
                                   stream=stream)
            g.gpcg_solve(dp, do)
            best = None
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g.gpcg_solve(dp, do)
                e1.record(stream)
                e1.synchronize()
                t = e0.elapsed_time(e1)
                best = t if best is None else min(best, t)
            xd, sd = g.gpcg_result(dp)
            row[name] = {"ms": best, "cg_iters": sd["cg_iters"], "passes": sd["passes"],
                         "alg_GB": sd["alg_bytes"] / 1e9}
        row["free_fraction"] = float(np.mean(xd > 0))
        ablation[f"disc_{frac}"] = row
        del dp, dqp

    # end to end through the C ABI from pinned host buffers
    pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(qp, k))).pin_memory()
           for k in ("diag", "cx", "cy", "b", "l", "u")}
    xh = torch.empty(qp.n, dtype=torch.float64).pin_memory()
    h2d = sum(t.numel() * 8 for t in pin.values())
    d2h = xh.numel() * 8
    # (a stream of QPs of one shape: two problems are created once and used
    # in turn; each step's data are copied in on a copy stream while the
    # previous step's QP is solved, then the step's QP is solved and x read
    # back)
    opts = g.default_options(tau_rel=TAU_REL, precision=g.MIXED, stream=stream)
    copy_stream = torch.cuda.Stream()
    pq = [g.gpcg_problem_create(dim=2, nx=qp.nx, ny=qp.ny, **pin) for _ in range(2)]

    def e2e_run(n_steps):
        g.gpcg_problem_update_async(pq[0], **pin, stream=copy_stream)
        for k in range(n_steps):
            if k + 1 < n_steps:
                g.gpcg_problem_update_async(pq[(k + 1) % 2], **pin, stream=copy_stream)
            g.gpcg_solve(pq[k % 2], opts)
            g.gpcg_result(pq[k % 2], xh)

    e2e_run(3)
    torch.cuda.synchronize()
    _barrier(ws)
    e_steps = max(1, min(args.steps, 30))
    t0 = time.perf_counter()
    e2e_run(e_steps)
    torch.cuda.synchronize()
    del pq
    e2e_t = _max_over_ranks(ws, time.perf_counter() - t0)
    e2e = {"value": ws * e_steps / e2e_t, "unit": "solves/s", "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h}

    # the small single QP (32 x 32, tau_rel 1e-8: latency-bound) and the 3-D
    # precision-stress QP (128^3 7-point, anisotropic): latency and solves/s,
    # and how far the mixed result is from the FP64 one
    small = {}
    sq = gi.single_small()
    sp = g.gpcg_problem_create(sq)
    # the resident solver (taken by default at this size) and the pass engine
    for name, prec, path in (("mixed", g.MIXED, g.PATH_AUTO), ("fp64", g.FP64, g.PATH_AUTO),
                             ("mixed_engine", g.MIXED, g.PATH_ENGINE),
                             ("fp64_engine", g.FP64, g.PATH_ENGINE)):
        so = g.default_options(tau_rel=1e-8, precision=prec, stream=stream, path=path)
        for _ in range(3):
            g.gpcg_solve(sp, so)
        ms = []
        for _ in range(50):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.gpcg_solve(sp, so)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        ms.sort()
        _, ss = g.gpcg_result(sp)
        small[name] = {"p50_ms": ms[len(ms) // 2], "p99_ms": ms[min(len(ms) - 1, int(0.99 * len(ms)))],
                       "solves/s": 1000.0 * len(ms) / sum(ms), "passes": ss["passes"],
                       "status": ss["status"],
                       "solver": "resident" if ss["path"] == g.PATH_RESIDENT else "engine",
                       "cg_iters": ss["cg_iters"], "gp_iters": ss["gp_iters"]}
    small["n"] = sq.n
    del sp
    stress = {}
    cq = gi.precision_stress()
    cp = g.gpcg_problem_create(cq)
    xs = {}
    for name, prec, rf in (("mixed", g.MIXED, 2), ("fp64", g.FP64, 2),
                           ("mixed_refine1", g.MIXED, 1)):
        co = g.default_options(tau_rel=TAU_REL, precision=prec, stream=stream, refine=rf)
        g.gpcg_solve(cp, co)
        ms = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.gpcg_solve(cp, co)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        xs[name], cs = g.gpcg_result(cp)
        stress[name] = {"solves/s": 1000.0 * len(ms) / sum(ms), "ms": min(ms),
                        "passes": cs["passes"], "cg_iters": cs["cg_iters"],
                        "pg_norm": cs["pg_norm"], "tau": cs["tau"], "status": cs["status"]}
    stress["n"] = cq.n
    stress["mixed_vs_fp64_rel_err"] = float(np.linalg.norm(xs["mixed"] - xs["fp64"]) /
                                            np.linalg.norm(xs["fp64"]))
    # the error against the FP64 oracle's solution at tau_rel 1e-12 (stored,
    # sampled at 65,536 points: tests/golden/precision_stress_128_oracle.npz)
    golden = os.path.join(ROOT, "tests", "golden", "precision_stress_128_oracle.npz")
    if os.path.exists(golden):
        gd = np.load(golden)
        idx = gd["idx"]
        for name in ("mixed", "fp64", "mixed_refine1"):
            stress[name]["max_err_vs_oracle_sampled"] = float(
                np.max(np.abs(xs[name][idx] - gd["x_sample"])) / max(1.0, float(gd["x_inf"])))
        stress["oracle_reference"] = (f"oracle at tau_rel {float(gd['tau_rel']):g}, "
                                      f"{idx.size} sampled points; the GPU solves above stop "
                                      f"at tau_rel {TAU_REL:g}")
    del cp, cq, xs

    batched = bench_batched(g, stream) if args.serve_seconds > 0 else None
    serving = bench_serving(g, args.serve_seconds) if args.serve_seconds > 0 else None

    if rank != 0:
        return
    cpu = cpu_baseline(qp) if ws == 1 else None
    lat = sorted(ms_mx)
    p = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
    line = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sum(ms_mx) / len(ms_mx), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32-stream/f64-reduce", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": qp.n, "grid": [qp.nx, qp.ny], "tau_rel": TAU_REL,
                   "parallelism": f"replicas{ws}",
                   "l2": "working set 0.43 GB > 129 MB L2 (inputs larger than L2)"},
        "p50_ms": p(0.5), "p99_ms": p(0.99),
        "fp64": {"value": value_64, "unit": "solves/s",
                 "ms_per_step": sum(ms_64) / len(ms_64), "roofline": roof_64,
                 "clocks": clk_64,
                 "solve": {k: st_64[k] for k in ("outer_iters", "gp_iters", "cg_iters",
                                                 "ls_trials", "passes", "pg_norm", "tau")}},
        "mixed_over_fp64": value / value_64,
        "mixed_refine1": {"value": ws * len(ms_r1) / _max_over_ranks(ws, sum(ms_r1) / 1000.0),
                          "unit": "solves/s", "ms_per_step": sum(ms_r1) / len(ms_r1),
                          "roofline": roof(ms_r1, st_r1, None),
                          "solve": {k: st_r1[k] for k in ("outer_iters", "gp_iters", "cg_iters",
                                                          "refine_cg_iters", "passes",
                                                          "pg_norm", "tau")}},
        "jacobi": jac,
        "tile": tile,
        "journal_bearing_1600": jb,
        "cg_system_1600_mixed": ablation,
        "single_small_32": small,
        "precision_stress_128": stress,
        "batched_512": batched,
        "serving": serving,
        "roofline": roof_mx,
        "spmv": spmv,
        "solve": {k: st_mx[k] for k in ("outer_iters", "gp_iters", "cg_iters", "ls_trials",
                                        "refine_cg_iters", "passes", "pg_norm", "tau",
                                        "n_active", "n_free")},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(args.steps * st_mx["launches"]),
        "clocks": clk_mx,
    }
    print(json.dumps(line), flush=True)


def run_profile(args):
    """Small fixed workloads for profiler captures: `solve` runs `--steps`
    solves of the benchmark QP (`solve3d`: of the 3-D precision-stress QP,
    side `--side`), `spmv` a few launches of the masked product
    alone (L2 flushed before each), `spmv_stream` `--steps` rounds of
    back-to-back products over 6 distinct problems of the same shape."""
    import torch
    import paper_cs_0101018_gb300 as g
    prec = g.MIXED if args.precision == "mixed" else g.FP64
    pc = {"none": g.PRECOND_NONE, "jacobi": g.PRECOND_JACOBI, "tile": g.PRECOND_TILE}[args.precond]
    qp = gi.precision_stress(args.side) if args.profile == "solve3d" else gi.single_large(args.side)
    prob = g.gpcg_problem_create(qp)
    if args.profile in ("solve", "solve3d"):
        for _ in range(args.steps):
            g.gpcg_solve(prob, g.default_options(tau_rel=TAU_REL, precision=prec, precond=pc))
        _, st = g.gpcg_result(prob)
        print(json.dumps({"profile": args.profile, "precision": args.precision,
                          "passes": st["passes"], "launches": st["launches"],
                          "cg_iters": st["cg_iters"]}))
    elif args.profile == "spmv_stream":
        probs = [prob] + [g.gpcg_problem_create(gi.grid_qp_2d(qp.nx, qp.ny, seed=sd, shift=1e-3,
                                                              bounds="two_sided"))
                          for sd in (11, 12, 13, 14, 15)]
        ms, by = g.gpcg_time_masked_spmv_stream(probs, prec, reps=args.steps)
        print(json.dumps({"profile": "spmv_stream", "precision": args.precision, "us": 1000 * ms,
                          "GB/s": by / ms / 1e6}))
    else:
        ms, by = g.gpcg_time_masked_spmv(prob, prec, reps=args.steps, flush_l2=True)
        print(json.dumps({"profile": "spmv", "precision": args.precision, "us": 1000 * ms,
                          "GB/s": by / ms / 1e6}))
    torch.cuda.synchronize()


def run_serve(args):
    """The batched and serving workloads alone (the full 60-s trace with
    `--serve-seconds 60`)."""
    import torch
    import paper_cs_0101018_gb300 as g
    stream = torch.cuda.Stream()
    print(json.dumps({"batched_512": bench_batched(g, stream),
                      "serving": bench_serving(g, args.serve_seconds)}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--profile", choices=["solve", "solve3d", "spmv", "spmv_stream", "serve"],
                    default=None,
                    help="run a small fixed workload for a profiler capture instead")
    ap.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    ap.add_argument("--precond", choices=["none", "jacobi", "tile"], default="none",
                    help="preconditioner of the CG phase (profile workloads only)")
    ap.add_argument("--side", type=int, default=1600,
                    help="grid side of the profile workloads (the benchmark QP at 1600)")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="length of the serving trace replayed (the full trace is 60 s; 0 "
                         "skips the batched and serving workloads)")
    args = ap.parse_args()
    if args.profile == "serve":
        run_serve(args)
    elif args.profile:
        run_profile(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
