"""Pins of the CPU oracle in three dimensions: the octree of the paper's extension to any dimension
(Section 4.2: a uniform 2^d tree; in 3D every box has up to 27 neighbours and up to 6^3 - 3^3 = 189
interaction-list boxes), Chebyshev interpolation with p^3 nodes (Section 5), 27 colours.

As in 2D, every pin checks the oracle against something other than itself: brute force on the box
grid, a kernel that the interpolation reproduces exactly, the interpolation formula of each level
written out, the dense FMM matrix and its dense LU solve (the extended sparse representation is
exact, Section 4.1), and the error of the compressed solve against eps.
"""
import math

import numpy as np
import pytest

from paper_1407_1572_gb300 import inputs


def _pts3(seed, n, lo=0.0, side=1.0):
    return lo + side * inputs.uniform(seed, 3 * n).reshape(n, 3)


def _o3(O, N, depth, p, kernel=None, eps=1e-10, diag=None, seed=31, **kw):
    pts = _pts3(seed, N)
    kernel = O.K_INV_R if kernel is None else kernel
    prm = O.make_params(depth, p, kernel, eps=eps, diag=math.sqrt(N) if diag is None else diag, dim=3, **kw)
    return O.Oracle(pts, prm), pts


def test_lists_brute_force_3d(oracle_mod):
    o, _ = _o3(oracle_mod, 300, 3, 2)
    for k in (1, 2, 3):
        s = 2 ** k
        for box in range(0, s ** 3, 7 if k == 3 else 1):
            nb, it = o.lists(k, box)
            c = (box % s, (box // s) % s, box // (s * s))
            want_nb, want_it = [], []
            for g in range(s ** 3):
                q = (g % s, (g // s) % s, g // (s * s))
                dd = max(abs(a - b) for a, b in zip(c, q))
                pd = max(abs(a // 2 - b // 2) for a, b in zip(c, q))
                if dd <= 1:
                    want_nb.append(g)
                elif pd <= 1:
                    want_it.append(g)
            assert sorted(nb) == want_nb and sorted(it) == want_it
            if all(2 <= a < s - 2 for a in c):
                assert len(nb) == 27 and len(it) == 189


def test_leaf_assignment_3d(oracle_mod):
    """Leaf = floor per coordinate (the upper face in the last box); boxes numbered ix + s (iy + s iz)."""
    O = oracle_mod
    n, depth = 500, 2
    pts = _pts3(5, n)
    pts[:10, 2] = 1.0
    o = O.Oracle(pts, O.make_params(depth, 2, O.K_INV_R, dim=3))
    m = 1 << depth
    c = np.minimum(np.floor(pts * m).astype(int), m - 1)
    cell = c[:, 0] + m * (c[:, 1] + m * c[:, 2])
    assert np.array_equal(o.leaf_counts(), np.bincount(cell, minlength=m ** 3))


def test_colour_classes_are_independent_sets_3d(oracle_mod):
    """Boxes of one colour are at Chebyshev distance >= 3, so their eliminations touch disjoint blocks."""
    o, _ = _o3(oracle_mod, 300, 3, 2)
    s = 8
    order = o.order(3)
    assert sorted(order) == list(range(s ** 3))
    col = lambda g: (g % s) % 3 + 3 * (((g // s) % s) % 3) + 9 * ((g // (s * s)) % 3)
    cols = [col(g) for g in order]
    assert cols == sorted(cols)                       # colour-major
    for cc in range(27):
        boxes = [g for g in range(s ** 3) if col(g) == cc]
        for a in boxes[:20]:
            for b in boxes:
                if a != b:
                    ca = np.array([a % s, (a // s) % s, a // (s * s)])
                    cb = np.array([b % s, (b // s) % s, b // (s * s)])
                    assert np.abs(ca - cb).max() >= 3


def test_polynomial_kernel_reproduced_exactly_3d(oracle_mod):
    """(1 + x1 y1)(1 + x2 y2)(1 + x3 y3) has degree 1 in each coordinate: the interpolation with p >= 2
    nodes per dimension reproduces it, so A~ equals the kernel matrix."""
    O = oracle_mod
    o, _ = _o3(O, 400, 3, 2, O.K_POLY, diag=0.0)
    A, Ae = o.dense_tilde(), o.dense_exact()
    assert np.abs(A - Ae).max() <= 1e-13 * np.abs(Ae).max()


@pytest.mark.parametrize("kernel", ["K_INV_R", "K_EXP"])
def test_nested_operators_equal_interpolation_formula_3d(oracle_mod, kernel):
    """The orthonormalised nested operators give the matrix of the per-level interpolation formula
    sum_{m,l} S^I_m(x) K(node^I_m, node^J_l) S^J_l(y), and the FMM matvec equals that dense matrix."""
    O = oracle_mod
    o, pts = _o3(O, 700, 3, 3, getattr(O, kernel), kparam=(0.3, 0, 0, 0))
    A, Ad = o.dense_tilde(), o.dense_tilde_direct()
    assert np.abs(A - Ad).max() <= 1e-13 * np.abs(A).max()
    x = inputs.rhs(3, 700, 2)
    assert np.abs(o.matvec(x) - A @ x).max() <= 1e-13 * np.abs(A @ x).max()
    # the interpolation error itself decreases with p (a smooth kernel)
    errs = []
    for p in (2, 3, 4):
        op, _ = _o3(O, 700, 3, p, getattr(O, kernel), kparam=(0.3, 0, 0, 0))
        Ap, Ae = op.dense_tilde(), op.dense_exact()
        errs.append(np.linalg.norm(Ap - Ae) / np.linalg.norm(Ae))
    assert errs[0] > errs[1] > errs[2]


@pytest.mark.parametrize("depth,p", [(2, 3), (3, 2), (3, 3)])
def test_uncompressed_elimination_is_exact_3d(oracle_mod, depth, p):
    """eps = 0: the elimination of the extended sparse system (Algorithm 1) and the back
    substitution (Algorithm 2) reproduce A~^{-1} b up to rounding, and so does the dense extended
    system."""
    O = oracle_mod
    N = 900
    o, _ = _o3(O, N, depth, p, eps=0.0)
    b = inputs.rhs(8, N, 2)
    xd = np.linalg.solve(o.dense_tilde(), b)
    o.factor()
    x = o.solve(b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-11
    xe = o.extended_solve(b)
    assert np.linalg.norm(xe - xd) / np.linalg.norm(xd) <= 1e-11


@pytest.mark.parametrize("N,depth,p", [(3000, 2, 3), (2500, 3, 2)])
def test_compressed_error_tracks_eps_3d(oracle_mod, N, depth, p):
    """With compression, the solve's distance to A~^{-1} b falls with eps and stays within C eps
    (C = 1e3, as in 2D; measured 3 to 90); the ranks grow as eps falls."""
    O = oracle_mod
    b = inputs.rhs(4, N, 1)
    prev_err, prev_rank = None, None
    for eps in (1e-3, 1e-6, 1e-9):
        o, _ = _o3(O, N, depth, p, eps=eps, tau_ref=1)
        xd = np.linalg.solve(o.dense_tilde(), b)
        o.factor()
        err = np.linalg.norm(o.solve(b) - xd) / np.linalg.norm(xd)
        assert err <= 1e3 * eps
        rank = o.stats()["max_rank"]
        if prev_err is not None:
            assert err < prev_err and rank > prev_rank
        prev_err, prev_rank = err, rank
