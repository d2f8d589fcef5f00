"""How far rounding alone moves a compressed IFMM solution at the parity workloads' sizes: the
reason the GPU's FP64 parity gates above 9,001 points are looser than 1e-10.

The oracle is run twice on 65,536 uniform points (depth 5, eps 1e-6, matrix-scale threshold,
1/r + sqrt(N) I): once on the points, once on the points with the last bit of every coordinate
flipped (a relative change of 2^-52, less than the rounding of any kernel evaluation). The two
solutions differ by about 1e-9 (rank 16) and 1.5e-8 (rank 36), element-wise relative to the
largest element, with identical ranks. Two mechanisms: the system is indefinite and the pivot
blocks reach condition numbers near 1e7, so a rounding-level change of the input moves the
fill-ins by about 1e-9 of their size; and the pivoted Gram-Schmidt of the compression (reading R2)
chooses each pivot by comparing column norms, so where two candidates are that close a different
column, hence a different remainder below the threshold, is kept. Any two FP64 codes whose
roundings differ (the GPU's Gauss-Jordan inverses and tiled sums, the oracle's LU solves and
sequential sums) differ by this much; 1e-10 is out of reach at these sizes."""
import math

import numpy as np
import pytest

from paper_1407_1572_gb300 import inputs


@pytest.mark.parametrize("p,lo,hi", [(4, 3e-10, 1e-8), (6, 3e-9, 1e-7)])
def test_one_ulp_of_the_points_moves_the_solution_beyond_1e_10(oracle_mod, p, lo, hi):
    O = oracle_mod
    N, depth = 65536, 5
    pts = inputs.uniform_points(1407 + N, N)
    flip = np.where(inputs.rhs(10, N, 2) >= 0.0, 1.0, -1.0)
    ptsp = np.clip(pts * (1.0 + 2.0 ** -52 * flip), 0.0, 1.0)
    b = inputs.rhs(9, N, 1)
    xs, ranks = [], []
    for P in (pts, ptsp):
        o = O.Oracle(P, O.make_params(depth, p, O.K_INV_R, eps=1e-6, diag=math.sqrt(N), tau_ref=1))
        o.factor()
        xs.append(o.solve(b))
        ranks.append([o.ranks(k) for k in range(2, depth + 1)])
    d = float(np.abs(xs[0] - xs[1]).max() / np.abs(xs[0]).max())
    assert all(np.array_equal(a, c) for a, c in zip(*ranks))
    assert lo <= d <= hi, d
