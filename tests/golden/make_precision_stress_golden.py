"""Writes precision_stress_128_oracle.npz: the oracle's solution of the 128^3
precision-stress QP (3-D 7-point, axis weights (1, 10, 100) x lognormal(0,1),
shift 4e-3, b ~ N(0,1), l = -1, u = 1, seed 4; gpcg_inputs.precision_stress)
at tau_rel 1e-12, for the full-size parity test of that workload.

The full solution is 2.1e6 doubles; the file keeps what the test compares:
  * x at 65,536 points drawn once (seeded, counter-based: gpcg_inputs.uniform,
    seed 44, stream 1), compared element by element;
  * the active set A(x) = {x_i = l_i or x_i = u_i} and the points within 1e-8
    of a bound, as packed bit masks of all n points;
  * ||x||_inf, ||x||_2, q(x) and the oracle's statistics;
  * a fingerprint of the QP's arrays (per array: sum, sum of squares and three
    entries), so that a change of the generator is seen.  The generator's
    transcendental functions (numpy's exp, log, cos) may differ in the last
    bit between hosts, so the fingerprint is compared with a relative
    tolerance of 1e-12, not bit for bit; inputs that close move the solution
    by about the condition number (1e5) times that, far inside the 1e-9
    parity tolerance.

This script calls only the oracle (oracle/) and the seeded input generators
(gpcg_inputs); it takes about ten minutes on eight cores.

    python tests/golden/make_precision_stress_golden.py
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import gpcg_inputs as gi  # noqa: E402
import oracle  # noqa: E402

OUT = os.path.join(HERE, "precision_stress_128_oracle.npz")
TAU_REL = 1e-12
SAMPLES = 65536
BAND = 1e-8


def qp_fingerprint(qp) -> np.ndarray:
    """Per array of the QP (diag, cx, cy, cz, b, l, u): the sum, the sum of
    squares and the entries at 0, n/2 and n-1."""
    out = []
    for a in (qp.diag, qp.cx, qp.cy, qp.cz, qp.b, qp.l, qp.u):
        a = np.ascontiguousarray(a, dtype=np.float64)
        out += [float(np.sum(a)), float(np.dot(a, a)), a[0], a[a.size // 2], a[-1]]
    return np.array(out)


def fingerprint_matches(fp_now, fp_stored, rtol: float = 1e-12) -> bool:
    return bool(np.allclose(fp_now, fp_stored, rtol=rtol, atol=0.0))


def sample_indices(n: int) -> np.ndarray:
    return np.unique((gi.uniform(44, 1, SAMPLES) * n).astype(np.int64)).astype(np.int64)


def main() -> None:
    qp = gi.precision_stress()
    oracle.set_threads(0)
    t0 = time.time()
    r = oracle.solve(qp, tau_rel=TAU_REL)
    dt = time.time() - t0
    assert r.status == oracle.OK, r.stats
    x = r.x
    idx = sample_indices(qp.n)
    active = (x == qp.l) | (x == qp.u)
    near = (np.abs(x - qp.l) <= BAND) | (np.abs(x - qp.u) <= BAND)
    np.savez_compressed(
        OUT, tau_rel=TAU_REL, n=qp.n, fingerprint=qp_fingerprint(qp), idx=idx, x_sample=x[idx],
        active=np.packbits(active), near=np.packbits(near), x_inf=float(np.max(np.abs(x))),
        x_norm2=float(np.linalg.norm(x)), q=float(r.stats["q"]),
        pg_norm=float(r.stats["pg_norm"]), pg_norm0=float(r.stats["pg_norm0"]),
        stats=np.array([r.stats[k] for k in ("outer_iters", "gp_iters", "cg_iters",
                                               "ls_trials", "n_active", "n_binding")]),
        oracle_seconds=dt, threads=oracle.threads())
    print(OUT, dt, r.stats)


if __name__ == "__main__":
    main()
