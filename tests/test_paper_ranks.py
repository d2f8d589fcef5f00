"""The paper's rank table for its benchmark kernels (Table "table_numerical_ranks_2D", stored in
tests/golden/ranks_2d_table.txt) against the oracle's kernels.

The paper does not state where the particles sit inside the clusters; the reading here is three
unit squares side by side with the N = m^2 particles of each on the cell centres of an m x m grid
(the printed N are squares). On that geometry the numbers do not reproduce exactly (measured: the
well-separated and Schur-complement ranks 1.2-1.6x the printed ones, the neighbour ranks growing
faster), so the test checks what the table is printed to show, with the printed values as scale:
(1) the well-separated ranks, before and after the Schur complement, stay within a factor 2 of the
printed ones and below the neighbour rank; (2) from N = 64 to N = 441 the Schur complement's rank
grows more slowly than the neighbour rank, the property the elimination's compression relies on.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ranks_2d_table.txt")
KERNELS = {"log_reg": O.K_LOG_REG, "inv_reg": O.K_INV_REG, "r2log_reg": O.K_R2LOG_REG}


def _table():
    rows = {}
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            k, n, g12, g13, s = line.split()
            rows[(k, int(n))] = (int(g12), int(g13), int(s))
    return rows


def _cluster(m, x0):
    t = (np.arange(m) + 0.5) / m
    X, Y = np.meshgrid(t + x0, t)
    return np.stack([X.ravel(), Y.ravel()], 1)


def _rank(A):
    s = np.linalg.svd(A, compute_uv=False)
    return int((s >= 1e-15 * s[0]).sum())


def _ranks(kernel, m):
    prm = O.make_params(2, 2, KERNELS[kernel], kparam=(0.005, 0, 0, 0))
    c1, c2, c3 = _cluster(m, 0.0), _cluster(m, 1.0), _cluster(m, 2.0)
    G12, G13 = O.kernel_matrix(prm, c1, c2), O.kernel_matrix(prm, c1, c3)
    G22, G23 = O.kernel_matrix(prm, c2, c2), O.kernel_matrix(prm, c2, c3)
    S = G13 - G12 @ np.linalg.solve(G22, G23)
    return _rank(G12), _rank(G13), _rank(S)


def test_golden_table_is_complete():
    t = _table()
    assert len(t) == 21 and all(k in KERNELS for k, _ in t)


@pytest.mark.parametrize("kernel", sorted(KERNELS))
def test_well_separated_ranks_stay_low_after_the_schur_complement(kernel):
    table = _table()
    got = {m * m: _ranks(kernel, m) for m in (8, 11, 15, 21)}
    for n, (g12, g13, s) in got.items():
        p12, p13, ps = table[(kernel, n)]
        assert g13 <= 2 * p13 and s <= 2 * ps, (n, (g12, g13, s), (p12, p13, ps))
        assert g13 < g12 and s < g12, (n, g12, g13, s)
    growth_s = got[441][2] / got[64][2]
    growth_nb = got[441][0] / got[64][0]
    assert growth_s < growth_nb, (kernel, growth_s, growth_nb)


def test_kernel_matrix_equals_pointwise_values():
    prm = O.make_params(2, 2, O.K_R2LOG_REG, kparam=(0.005, 0, 0, 0))
    P, Q = _cluster(3, 0.0), _cluster(2, 0.0015)
    M = O.kernel_matrix(prm, P, Q)
    for i in range(len(P)):
        for j in range(len(Q)):
            assert M[i, j] == O.kernel_eval(prm, P[i], Q[j])
