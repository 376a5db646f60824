"""The journal bearing workload of Sec. 5 (finite-difference form, see
gpcg_inputs.journal_bearing): properties of the generated QP and the
oracle's solution; the paper's finite-element numbers are matched only
qualitatively (free fraction at the solution ~68 % for eps = 0.1 and ~54 %
for eps = 0.9, decreasing with eps)."""
import numpy as np
import pytest

import gpcg_inputs as gi
import oracle
from oracle import brute_force as bf


@pytest.mark.parametrize("eps", [0.1, 0.9])
def test_generator_is_an_m_matrix_with_the_bearing_load(eps):
    qp = gi.journal_bearing(23, 17, eps)
    A = bf.dense_matrix(qp)
    assert np.allclose(A, A.T)
    off = A - np.diag(np.diag(A))
    assert np.all(off <= 0)  # couplings are negative edge weights
    row = np.diag(A) + off.sum(axis=1)  # diag - sum |off|: the boundary edges
    assert np.all(row >= -1e-12) and np.any(row > 1e-6)
    assert np.linalg.eigvalsh(A).min() > 0
    xi1 = (np.arange(qp.n) % qp.nx + 1) * qp.meta["h1"]
    assert np.all(qp.b[xi1 < np.pi - 1e-9] < 0) and np.all(qp.b[xi1 > np.pi + 1e-9] > 0)
    # w_q is largest where the film is thickest (xi_1 near 0 and 2 pi)
    assert qp.diag[0] > qp.diag[qp.nx // 2]


def test_oracle_solution_free_fraction_and_kkt():
    free = {}
    for eps in (0.1, 0.9):
        qp = gi.journal_bearing(60, 40, eps)
        r = oracle.solve(qp, tau_abs=1e-11, tau_rel=0.0)
        assert r.status == oracle.OK
        A = bf.dense_matrix(qp)
        assert bf.kkt_residual(A, qp.b, qp.l, qp.u, r.x) < 1e-9
        assert np.all(r.x >= 0)
        free[eps] = float(np.mean(r.x > 0))
    assert 0.60 < free[0.1] < 0.75 and 0.45 < free[0.9] < 0.60
    assert free[0.1] > free[0.9]
