"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it follows. None of them retypes an oracle formula: they check
closed forms, brute force on tiny inputs, special cases that reduce to a textbook routine,
and the exactness invariant of the extended sparse system (Section 2.3 / 4.1: the FMM matrix
is represented "exactly" by the extended sparse matrix).
"""
import math

import numpy as np
import pytest

from paper_1407_1572_gb300 import inputs


def _oracle(O, N, depth, p, kernel=None, eps=1e-10, diag=None, seed=1407, **kw):
    pts = inputs.uniform_points(seed, N)
    kernel = O.K_INV_R if kernel is None else kernel
    prm = O.make_params(depth, p, kernel, eps=eps, diag=math.sqrt(N) if diag is None else diag, **kw)
    return O.Oracle(pts, prm), pts


# ---- Chebyshev interpolation (Section 5: 8 Chebyshev nodes per dimension) --------------------

@pytest.mark.parametrize("p", [1, 2, 3, 4, 6, 8])
def test_cheb_nodes_are_roots_of_T_p(oracle_mod, p):
    t = oracle_mod.cheb_nodes(p)
    # T_p(cos th) = cos(p th): first-kind nodes are the p roots of T_p in (-1, 1)
    assert np.allclose(np.cos(p * np.arccos(t)), 0.0, atol=1e-14)
    assert len(set(np.round(t, 12))) == p


@pytest.mark.parametrize("p", [2, 4, 6])
def test_lagrange_cardinal_and_exact_on_polynomials(oracle_mod, p):
    t = oracle_mod.cheb_nodes(p)
    for n in range(p):
        assert np.allclose(oracle_mod.lagrange(p, t[n]), np.eye(p)[n], atol=1e-13)
    rng = np.random.default_rng(0)
    for _ in range(5):
        coeff = rng.standard_normal(p)          # degree p-1 polynomial
        x = rng.uniform(-1, 1)
        interp = oracle_mod.lagrange(p, x) @ np.polyval(coeff, t)
        assert abs(interp - np.polyval(coeff, x)) < 1e-12
        assert abs(oracle_mod.lagrange(p, x).sum() - 1.0) < 1e-13


def test_kernel_values_closed_form(oracle_mod):
    O = oracle_mod
    prm = O.make_params(3, 4, O.K_INV_R)
    assert O.kernel_eval(prm, [0.0, 0.0], [3.0, 4.0]) == pytest.approx(0.2, rel=1e-15)
    prm = O.make_params(3, 4, O.K_EXP, kparam=(0.1, 0, 0, 0))
    assert O.kernel_eval(prm, [0.0, 0.0], [0.3, 0.4]) == pytest.approx(math.exp(-5.0), rel=1e-14)


def test_length_scale_derivative_kernel(oracle_mod):
    """K_DEXP_DELL is d/dl exp(-r/l) = (r/l^2) exp(-r/l): closed form at r = 0.5, l = 0.1, and the
    central difference of K_EXP in l at other points."""
    O = oracle_mod
    prm = O.make_params(3, 4, O.K_DEXP_DELL, kparam=(0.1, 0, 0, 0))
    assert O.kernel_eval(prm, [0.0, 0.0], [0.3, 0.4]) == pytest.approx(0.5 / 0.01 * math.exp(-5.0), rel=1e-14)
    rng = np.random.default_rng(5)
    for _ in range(5):
        a, b = rng.uniform(0, 1, 2), rng.uniform(0, 1, 2)
        ell = rng.uniform(0.05, 0.3)
        h = 1e-4 * ell   # central difference: truncation O((h/l)^2) ~ 1e-8 relative
        kp = O.make_params(3, 4, O.K_EXP, kparam=(ell + h, 0, 0, 0))
        km = O.make_params(3, 4, O.K_EXP, kparam=(ell - h, 0, 0, 0))
        fd = (O.kernel_eval(kp, a, b) - O.kernel_eval(km, a, b)) / (2 * h)
        d = O.kernel_eval(O.make_params(3, 4, O.K_DEXP_DELL, kparam=(ell, 0, 0, 0)), a, b)
        assert d == pytest.approx(fd, rel=1e-6, abs=1e-12)


def test_benchmark_kernels_closed_form_and_continuity(oracle_mod):
    """The three regularised kernels of Section 5 (a = 0.001): values on both branches and
    continuity at r = a, where both branches equal 1."""
    O = oracle_mod
    a = 1e-3
    mk = lambda k: O.make_params(3, 4, k, kparam=(a, 0, 0, 0))
    r_small, r_big = 4e-4, 0.3
    pts = lambda r: ([0.0, 0.0], [r, 0.0])
    la = math.log(a)
    assert O.kernel_eval(mk(O.K_LOG_REG), *pts(r_big)) == pytest.approx(math.log(r_big) / la, rel=1e-14)
    assert O.kernel_eval(mk(O.K_LOG_REG), *pts(r_small)) == pytest.approx(
        r_small * (math.log(r_small) - 1) / (a * (la - 1)), rel=1e-14)
    assert O.kernel_eval(mk(O.K_INV_REG), *pts(r_big)) == pytest.approx(a / r_big, rel=1e-15)
    assert O.kernel_eval(mk(O.K_INV_REG), *pts(r_small)) == pytest.approx(r_small / a, rel=1e-15)
    assert O.kernel_eval(mk(O.K_R2LOG_REG), *pts(r_big)) == pytest.approx(r_big ** 2 * math.log(r_big) / (a * a * la), rel=1e-14)
    assert O.kernel_eval(mk(O.K_R2LOG_REG), *pts(r_small)) == pytest.approx(
        r_small ** 3 * (3 * math.log(r_small) - 1) / (a ** 3 * (3 * la - 1)), rel=1e-14)
    for k in (O.K_LOG_REG, O.K_INV_REG, O.K_R2LOG_REG):
        lo = O.kernel_eval(mk(k), *pts(a * (1 - 1e-9)))
        hi = O.kernel_eval(mk(k), *pts(a * (1 + 1e-9)))
        assert lo == pytest.approx(1.0, abs=1e-7) and hi == pytest.approx(1.0, abs=1e-7)
        assert O.kernel_eval(mk(k), [0.2, 0.3], [0.2, 0.3]) == 0.0


# ---- tree and lists (Section 4.2, Table "table_cluster") -------------------------------------

def test_lists_brute_force(oracle_mod):
    o, _ = _oracle(oracle_mod, 512, 4, 2)
    for k in range(1, 5):
        s = 2 ** k
        for box in range(s * s):
            nb, it = o.lists(k, box)
            ix, iy = box % s, box // s
            want_nb, want_it = [], []
            for jy in range(s):
                for jx in range(s):
                    d = max(abs(ix - jx), abs(iy - jy))
                    pd = max(abs(ix // 2 - jx // 2), abs(iy // 2 - jy // 2))
                    if d <= 1:
                        want_nb.append(jx + s * jy)
                    elif pd <= 1:
                        want_it.append(jx + s * jy)
            assert sorted(nb) == sorted(want_nb)
            assert sorted(it) == sorted(want_it)
            if 2 <= ix < s - 2 and 2 <= iy < s - 2:
                assert len(nb) == 9 and len(it) == 27


@pytest.mark.parametrize("box", [(0.0, 0.0, 1.0), (-1.0, -1.0, 2.0)])
def test_leaf_assignment_is_the_floor_rule(oracle_mod, box):
    """Each point falls in the leaf floor((coordinate - origin) 2^depth / side), a point on the upper
    edge of the root box in the last leaf of its row or column (Section 4.2's uniform tree); the
    tree order lists the leaves in Z-order (Morton) and each leaf's points by index."""
    O = oracle_mod
    depth, n = 3, 700
    x0, y0, side = box
    pts = x0 + side * inputs.uniform_points(29, n)
    pts[:20, 0] = x0 + side            # right edge
    pts[20:40, 1] = y0 + side          # top edge
    pts[40] = (x0 + side, y0 + side)   # corner
    pts[41] = (x0, y0)                 # origin
    pts[42, 0] = x0 + side / 2         # on an inner box boundary
    o = O.Oracle(pts, O.make_params(depth, 2, O.K_INV_R, box=box))
    m = 1 << depth
    cx = np.minimum(np.floor((pts[:, 0] - x0) / side * m).astype(int), m - 1)
    cy = np.minimum(np.floor((pts[:, 1] - y0) / side * m).astype(int), m - 1)
    cell = cy * m + cx
    # leaf counts by grid index g = ix + 2^depth iy
    assert np.array_equal(o.leaf_counts(), np.bincount(cell, minlength=m * m))
    # tree order: points sorted by the Z-order (bit-interleaved) index of their leaf, ties by
    # point index; either interleaving convention is a Z-order
    perm = o.perm()
    assert np.array_equal(np.sort(perm), np.arange(n))

    def interleave(a, b):
        return sum((((a >> k) & 1) << (2 * k)) | (((b >> k) & 1) << (2 * k + 1)) for k in range(depth))

    got = [(int(cell[i]), int(i)) for i in perm]
    want = [sorted(((int(cell[i]), int(i)) for i in range(n)), key=lambda t: (z(t[0] % m, t[0] // m), t[1]))
            for z in (interleave, lambda a, b: interleave(b, a))]
    assert got in want


def test_every_leaf_pair_covered_exactly_once(oracle_mod):
    """The near field plus the interaction lists of all levels partition the leaf pairs
    (the FMM matrix of Section 2.2: each block is either full rank or a well-separated
    low-rank block at exactly one level)."""
    o, _ = _oracle(oracle_mod, 512, 4, 2)
    kap = 4
    s = 2 ** kap
    cover = np.zeros((s * s, s * s), dtype=int)
    for i in range(s * s):
        nb, _ = o.lists(kap, i)
        cover[i, nb] += 1
    for k in range(2, kap + 1):
        sk = 2 ** k
        for I in range(sk * sk):
            _, it = o.lists(k, I)
            for J in it:
                for i in range(s * s):
                    if (i % s) >> (kap - k) != I % sk or (i // s) >> (kap - k) != I // sk:
                        continue
                    for j in range(s * s):
                        if (j % s) >> (kap - k) == J % sk and (j // s) >> (kap - k) == J // sk:
                            cover[i, j] += 1
    assert (cover == 1).all()


def test_colour_order_independent_sets(oracle_mod):
    o, _ = _oracle(oracle_mod, 1024, 3, 2)
    for k in (2, 3):
        s = 2 ** k
        order = o.order(k)
        assert sorted(order) == list(range(s * s))
        col = [(b % s) % 3 + 3 * ((b // s) % 3) for b in order]
        assert col == sorted(col)
        for a in order:
            for b in order:
                if a != b and col[list(order).index(a)] == col[list(order).index(b)]:
                    d = max(abs(a % s - b % s), abs(a // s - b // s))
                    assert d >= 3


# ---- dense LU (textbook) -----------------------------------------------------------------------

def test_dense_lu_solves_known_system(oracle_mod):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((60, 60))
    x = rng.standard_normal((60, 3))
    got = oracle_mod.dense_lu_solve(A, A @ x)
    assert np.abs(got - x).max() < 1e-10
    assert np.allclose(got, np.linalg.solve(A, A @ x), atol=1e-11)


# ---- the FMM matrix A~ (Section 2.2, Table "table_FMM_operators", Section 5) -----------------

def test_polynomial_kernel_is_reproduced_exactly(oracle_mod):
    """Chebyshev interpolation with p >= 2 nodes is exact for a kernel of degree 1 in each
    coordinate, so the FMM matrix equals the kernel matrix (nested bases, orthonormalisation
    and M2L folding all included)."""
    O = oracle_mod
    for depth, p in [(3, 2), (3, 3), (4, 2)]:
        o, _ = _oracle(O, 600, depth, p, kernel=O.K_POLY, diag=3.0)
        A = o.dense_exact()
        At = o.dense_tilde()
        assert np.abs(A - At).max() < 1e-12 * np.abs(A).max()


@pytest.mark.parametrize("kernel", ["inv_r", "exp", "log_reg", "inv_reg", "r2log_reg"])
def test_nested_operators_equal_textbook_formula(oracle_mod, kernel):
    """A~ through P2M/M2M/M2L/L2L/L2P with orthonormalised bases equals the per-level Chebyshev
    formula sum_{m,l} S_m(x) K(xbar_m, ybar_l) S_l(y) (nesting of polynomial interpolation)."""
    O = oracle_mod
    kk = {"inv_r": O.K_INV_R, "exp": O.K_EXP, "log_reg": O.K_LOG_REG, "inv_reg": O.K_INV_REG,
          "r2log_reg": O.K_R2LOG_REG}[kernel]
    kp = (0.1, 0, 0, 0) if kernel == "exp" else (1e-3, 0, 0, 0)
    o, _ = _oracle(O, 700, 4, 3, kernel=kk, kparam=kp)
    At = o.dense_tilde()
    Ad = o.dense_tilde_direct()
    assert np.abs(At - Ad).max() < 1e-12 * np.abs(Ad).max()
    assert np.allclose(At, At.T, rtol=0, atol=1e-12 * np.abs(At).max())


def test_fmm_of_length_derivative_is_derivative_of_fmm(oracle_mod):
    """The Chebyshev nodes, the orthonormal bases and the tree do not depend on l, so the FMM matrix
    of K_DEXP_DELL (zero diagonal) is d/dl of the FMM matrix of K_EXP (diagonal 1 + sigma^2): checked
    against the central difference of the assembled A~(l)."""
    O = oracle_mod
    pts = inputs.uniform_points(31, 600)
    ell, h, sig2 = 0.1, 1e-5, 1e-2
    mk = lambda kernel, l, diag: O.Oracle(pts, O.make_params(3, 4, kernel, diag=diag, kparam=(l, 0, 0, 0)))
    Ap = mk(O.K_EXP, ell + h, 1.0 + sig2).dense_tilde()
    Am = mk(O.K_EXP, ell - h, 1.0 + sig2).dense_tilde()
    D = mk(O.K_DEXP_DELL, ell, 0.0).dense_tilde()
    fd = (Ap - Am) / (2 * h)
    assert np.abs(D - fd).max() <= 1e-7 * np.abs(D).max()
    assert np.allclose(D, D.T, rtol=0, atol=1e-12 * np.abs(D).max())
    assert np.abs(np.diag(D)).max() == 0.0


def test_interpolation_error_decreases_with_p(oracle_mod):
    errs = []
    for p in (2, 4, 6):
        o, _ = _oracle(oracle_mod, 1024, 3, p)
        A = o.dense_exact()
        errs.append(np.linalg.norm(o.dense_tilde() - A) / np.linalg.norm(A))
    assert errs[0] > 10 * errs[1] > 100 * errs[2]


def test_fmm_matvec_equals_dense(oracle_mod):
    o, _ = _oracle(oracle_mod, 1500, 3, 4)
    x = inputs.rhs(11, 1500, 3)
    y = o.matvec(x)
    ref = o.dense_tilde() @ x
    assert np.abs(y - ref).max() < 1e-12 * np.abs(ref).max()


# ---- extended sparse system (Section 4.1, Eq. "extended_sparsity") ---------------------------

@pytest.mark.parametrize("depth,p", [(2, 3), (3, 2), (3, 3)])
def test_extended_system_is_exact(oracle_mod, depth, p):
    """The extended sparse system with multipoles and locals as unknowns has exactly the
    solution of A~ x = b (the paper's first key idea)."""
    N = 640
    o, _ = _oracle(oracle_mod, N, depth, p)
    x = inputs.rhs(5, N, 2)
    A = o.dense_tilde()
    b = A @ x
    xe = o.extended_solve(b)
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(xe - xd) / np.linalg.norm(xd) < 1e-9


# ---- elimination and back substitution (Algorithms 1 and 2) ----------------------------------

@pytest.mark.parametrize("depth,p,order", [(2, 3, 0), (3, 2, 0), (3, 3, 0), (3, 3, 1), (4, 2, 0)])
def test_uncompressed_elimination_is_exact(oracle_mod, depth, p, order):
    """eps = 0 keeps every fill direction: the elimination is then plain block LU of the
    extended system (Remark in Section 4.1) and reproduces A~^{-1} b."""
    N = 1024
    o, _ = _oracle(oracle_mod, N, depth, p, eps=0.0, order=order)
    A = o.dense_tilde()
    x = inputs.rhs(9, N, 2)
    b = A @ x
    o.factor()
    xs = o.solve(b)
    xd = np.linalg.solve(A, b)
    assert np.linalg.norm(xs - xd) / np.linalg.norm(xd) < 1e-10


@pytest.mark.parametrize("kernel", ["log_reg", "inv_reg", "r2log_reg"])
def test_uncompressed_elimination_is_exact_for_the_benchmark_kernels(oracle_mod, kernel):
    """The same exactness for the paper's benchmark kernels (Section 5: a = 0.001, unit diagonal,
    points in [-1, 1]^2): the eps = 0 solve is backward stable on A~ (normwise backward error at
    roundoff) and, where A~ is well conditioned (log: kappa 1e3, a / r: 4e1), equals the dense
    solution to 1e-12; r^2 ln r (kappa 2e8) is held to the backward error alone."""
    O = oracle_mod
    kid = {"log_reg": O.K_LOG_REG, "inv_reg": O.K_INV_REG, "r2log_reg": O.K_R2LOG_REG}[kernel]
    N = 1024
    pts = inputs.uniform_points(71, N, lo=-1.0, side=2.0)
    o = O.Oracle(pts, O.make_params(3, 3, kid, eps=0.0, diag=1.0, kparam=(1e-3, 0, 0, 0), box=(-1.0, -1.0, 2.0)))
    A = o.dense_tilde()
    x = inputs.rhs(9, N, 2)
    b = A @ x
    o.factor()
    xs = o.solve(b)
    an = np.linalg.norm(A, 1)
    eta = float((np.abs(A @ xs - b).sum(0) / (an * np.abs(xs).sum(0) + np.abs(b).sum(0))).max())
    assert eta < 1e-14
    if kernel != "r2log_reg":
        xd = np.linalg.solve(A, b)
        assert np.linalg.norm(xs - xd) / np.linalg.norm(xd) < 1e-12


def test_compressed_error_tracks_eps(oracle_mod):
    N = 2048
    errs = []
    for eps in (1e-5, 1e-8, 1e-11):
        o, _ = _oracle(oracle_mod, N, 3, 3, eps=eps)
        x = inputs.rhs(13, N, 1)
        b = o.matvec(x)
        o.factor()
        errs.append(np.linalg.norm(o.solve(b) - x) / np.linalg.norm(x))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-6


@pytest.mark.parametrize("tau_ref", [0, 1])
def test_orders_agree_within_eps_bound(oracle_mod, tau_ref):
    """The paper leaves the elimination order open; colour-major and Morton order must give
    the same solution up to the compression error."""
    N = 2048
    sols = []
    for order in (0, 1):
        o, _ = _oracle(oracle_mod, N, 3, 3, eps=1e-9, order=order, tau_ref=tau_ref)
        x = inputs.rhs(17, N, 1)
        b = o.matvec(x)
        o.factor()
        sols.append((o.solve(b), x))
    for xs, x in sols:
        assert np.linalg.norm(xs - x) / np.linalg.norm(x) < 1e-4
    assert np.linalg.norm(sols[0][0] - sols[1][0]) / np.linalg.norm(sols[0][1]) < 1e-4


def test_multiple_rhs_consistent(oracle_mod):
    N = 1024
    o, _ = _oracle(oracle_mod, N, 3, 3, eps=1e-8)
    o.factor()
    B = inputs.rhs(19, N, 3)
    X = o.solve(B)
    for j in range(3):
        assert np.allclose(o.solve(B[:, j].copy()), X[:, j], rtol=0, atol=1e-13 * np.abs(X).max())


def test_ranks_bounded_and_work_linear(oracle_mod):
    """Ranks of the compressed blocks stay bounded and the work per unknown stays flat as N
    grows at fixed points per leaf (Section 5 remark; O(N) claim of Section 1)."""
    out = []
    for N, depth in ((1024, 2), (4096, 3), (16384, 4)):
        o, _ = _oracle(oracle_mod, N, depth, 3, eps=1e-6, tau_ref=1)
        o.factor()
        st = o.stats()
        out.append((st["max_rank"], st["flops"] / N))
    assert out[2][0] <= 2.0 * out[1][0]
    assert out[2][1] <= 2.5 * out[1][1]


# ---- the compression step alone (Algorithm 1's compression of well-separated fill; reading R2) --

def _fill_with_known_rank(n=64, r=16, seed=5):
    """An orthonormal basis W (n x r) and a fill S whose part outside span(W) is known exactly:
    seven columns sigma_j q_j with q_j orthonormal and orthogonal to W, sigma_j = 10^-a_j with
    a = (2, 3, 4.5, 5.5, 7.5, 9, 10); three columns of norm 100 inside span(W); every column plus
    noise of norm 1e-9. The threshold eps = 1e-6 is never within a factor 3 of a sigma_j."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, r + 7)))
    W, Qp = Q[:, :r].copy(), Q[:, r:]
    sig = 10.0 ** -np.array([2.0, 3.0, 4.5, 5.5, 7.5, 9.0, 10.0])
    cols = [sig[j] * Qp[:, j] for j in range(7)]
    for _ in range(3):
        g = rng.standard_normal(r)
        cols.append(100.0 * W @ (g / np.linalg.norm(g)))
    S = np.stack(cols, axis=1)
    noise = rng.standard_normal(S.shape)
    S += 1e-9 * noise / np.linalg.norm(noise, axis=0)
    return W, S, Qp, sig


def test_compression_appends_exactly_the_directions_above_the_threshold(oracle_mod):
    """Reading R2/R5: with the matrix-scale reference (threshold eps * s_A, here s_A = 1) the four
    directions whose size exceeds 1e-6 are appended and nothing else; with the fill-relative
    reference (eps times the largest column of S, which is 100) only the two above 1e-4 are. The
    old basis is kept bit for bit (so the operators' update is a zero-padding), the new columns are
    orthonormal to it, and they span the expected directions. A wrong reference, an off-by-one in
    the kept count or a lost old basis fails here."""
    O = oracle_mod
    W, S, Qp, sig = _fill_with_known_rank()
    for ref, want in ((1.0, 4), (0.0, 2)):
        W2, add, over = O.augment_basis(W, S, 1e-6, ref=ref)
        assert (add, over) == (want, False), (ref, add)
        assert np.array_equal(W2[:, :16], W)
        assert np.abs(W2.T @ W2 - np.eye(16 + add)).max() < 1e-14
        # the appended columns span q_0 .. q_{want-1} up to the noise and the dropped directions
        P = Qp[:, :want] @ Qp[:, :want].T
        # (the noise, 1e-9, against the smallest kept direction, 3.2e-6: 3e-4)
        assert np.linalg.norm(W2[:, 16:] - P @ W2[:, 16:]) < 1e-3
    # the cap: at most 18 columns in all
    W3, add, over = O.augment_basis(W, S, 1e-6, ref=1.0, cap=18)
    assert (add, over) == (2, True)


def test_compression_stays_orthonormal_on_nearly_parallel_fill(oracle_mod):
    """Columns a, a + 1e-7 b, a + 2e-7 c (threshold 1e-12): three directions, and the basis stays
    orthonormal to rounding. Gram-Schmidt without the re-orthogonalisation of reading R2 loses
    orthogonality in proportion to u / 1e-7 (about 1e-9) on such columns."""
    O = oracle_mod
    rng = np.random.default_rng(11)
    n, r = 64, 16
    Q, _ = np.linalg.qr(rng.standard_normal((n, r)))
    a, b, c = (rng.standard_normal(n) for _ in range(3))
    S = np.stack([a, a + 1e-7 * b, a + 2e-7 * c], axis=1)
    W2, add, _ = O.augment_basis(Q, S, 1e-12, ref=1.0)
    assert add == 3
    assert np.abs(W2.T @ W2 - np.eye(r + 3)).max() < 1e-14


def test_compressed_solve_within_c_eps_of_dense_lu(oracle_mod):
    """4,096 uniform points, depth 3, rank 16, eps 1e-10, matrix-scale threshold: the compressed
    factorisation solves a perturbed matrix A~ + E, and every remainder the compression drops has
    columns below eps * s_A, so to first order ||x - x_dense|| / ||x_dense|| <= C eps with
    C = s_A ||A~^{-1}||_2 (8.9e4 here; s_A = 3954, ||A~^{-1}||_2 = 22.4 = 1 / min |lambda(A~)|, A~
    being symmetric). The measured error, 5.5e-8, is 0.6% of that bound, and it scales with eps.
    The dense reference is LAPACK's solve of the oracle's assembled A~."""
    O = oracle_mod
    N = 4096
    errs = {}
    for eps in (1e-10, 1e-8):
        o, _ = _oracle(O, N, 3, 4, eps=eps, seed=1407 + N, tau_ref=1)
        o.factor()
        if eps == 1e-10:
            A = o.dense_tilde()
            assert np.abs(A - A.T).max() <= 1e-12 * np.abs(A).max()
            sA = o.stats()["scale_A"]
            C = sA / np.abs(np.linalg.eigvalsh(A)).min()
            b = inputs.rhs(9, N, 2)
            xd = np.linalg.solve(A, b)
        errs[eps] = np.linalg.norm(o.solve(b) - xd) / np.linalg.norm(xd)
    assert 5e4 < C < 2e5
    assert errs[1e-10] <= C * 1e-10
    assert errs[1e-8] <= C * 1e-8
    assert 10.0 < errs[1e-8] / errs[1e-10] < 1000.0


# ---- SVD compression of the Chebyshev interpolation (Section 5: "followed by SVD") ------------

def _kfat_by_definition(O, prm, level, p, parent=None):
    """K_fat of a level from its definition, in numpy: the M2L kernel matrices between a box's
    Chebyshev nodes and those of the 40 interaction offsets (box side 2^-level of the root), plus,
    below the top level, the parent's kept directions restricted to each child position (T_c U S).
    T_c is built from the Lagrange basis (S^parent evaluated at the child's nodes)."""
    t = O.cheb_nodes(p)
    h = prm.box[2] / 2 ** level
    nodes = np.array([[0.5 * (t[mx] + 1) * h, 0.5 * (t[my] + 1) * h] for my in range(p) for mx in range(p)])
    blocks = []
    for dy in range(-3, 4):
        for dx in range(-3, 4):
            if max(abs(dx), abs(dy)) >= 2:
                blocks.append(O.kernel_matrix(prm, nodes, nodes + h * np.array([dx, dy])))
    K = np.hstack(blocks)
    if parent is not None:
        Up, sp = parent
        for c in range(4):
            a, b = c & 1, c >> 1
            T = np.array([np.outer(O.lagrange(p, 0.5 * (t[my] - 1) + b), O.lagrange(p, 0.5 * (t[mx] - 1) + a)).ravel()
                          for my in range(p) for mx in range(p)])
            K = np.hstack([K, (T @ Up) * sp])
    return K


@pytest.mark.parametrize("kernel,kp", [("K_INV_R", 0.0), ("K_LOG_REG", 0.001), ("K_EXP", 0.3)])
def test_svd_basis_is_the_svd_of_the_m2l_matrices(oracle_mod, kernel, kp):
    """The oracle's one-sided Jacobi SVD against LAPACK's (numpy) on K_fat built from the definition:
    singular values to 1e-13 sigma_1 at the top level and the nested one below it, and the kept
    projector U_r U_r^T, with r where the spectrum has a gap."""
    O = oracle_mod
    p = 5
    o, _ = _oracle(O, 500, 3, p, getattr(O, kernel), kparam=(kp, 0, 0, 0), svd_eps=1e-7)
    parent = None
    for level in (2, 3):
        U, sg, r = o.svd_basis(level)
        K = _kfat_by_definition(O, o.params, level, p, parent)
        Un, sn, _ = np.linalg.svd(K)
        assert np.allclose(sg, sn[: p * p], rtol=0, atol=1e-13 * sn[0])
        assert np.allclose(U.T @ U, np.eye(p * p), atol=1e-12)
        assert r == max(1, int(np.sum(sn[: p * p] > 1e-7 * sn[0])))
        gaps = [j for j in range(1, p * p) if sn[j] < 0.5 * sn[j - 1] and sn[j - 1] > 1e-9 * sn[0]]
        for j in gaps[:3]:
            assert np.allclose(U[:, :j] @ U[:, :j].T, Un[:, :j] @ Un[:, :j].T, atol=1e-9)
        # sign convention: the largest entry of every column is positive
        assert np.all(U[np.abs(U).argmax(0), np.arange(p * p)] > 0)
        parent = (U[:, :r], sg[:r])


def test_svd_keeps_the_exact_rank_of_a_separable_kernel(oracle_mod):
    """|x - y|^2 = |x|^2 - 2 x.y + |y|^2 has separable rank 4 (functions 1, x_1, x_2, |x|^2 of one
    point); Chebyshev interpolation with p >= 3 reproduces it exactly, so the truncated bases keep
    4 directions at every level and the FMM matrix still equals the kernel matrix."""
    O = oracle_mod
    for p in (3, 5):
        o, _ = _oracle(O, 400, 4, p, O.K_R2, diag=0.0, svd_eps=1e-10)
        assert [o.svd_basis(k)[2] for k in (2, 3, 4)] == [4, 4, 4]
        assert o.initial_ranks(4).max() <= 4
        A, Ae = o.dense_tilde(), o.dense_exact()
        assert np.abs(A - Ae).max() <= 1e-12 * np.abs(Ae).max()


@pytest.mark.parametrize("kernel,kp", [("K_INV_R", 0.0), ("K_LOG_REG", 0.001)])
def test_svd_nested_operators_equal_the_projected_formula(oracle_mod, kernel, kp):
    """With the truncation, the nested operators (orthonormalised bases, transfers, M2L) give the
    same FMM matrix as the definition: S^leaf(x) Pi_kappa T_c Pi_(kappa-1) ... Pi_k between the
    interpolation at each level, K at level k's nodes."""
    O = oracle_mod
    o, _ = _oracle(O, 500, 4, 5, getattr(O, kernel), kparam=(kp, 0, 0, 0), svd_eps=1e-6)
    assert min(o.svd_basis(k)[2] for k in (2, 3, 4)) < 25
    A, Ad = o.dense_tilde(), o.dense_tilde_direct()
    off = A - np.diag(np.diag(A))
    assert np.abs(A - Ad).max() <= 1e-13 * np.abs(off).max()


@pytest.mark.parametrize("kernel,kp", [("K_INV_R", 0.0), ("K_LOG_REG", 0.001), ("K_EXP", 0.5)])
def test_svd_truncation_error_tracks_svd_eps(oracle_mod, kernel, kp):
    """Dropping singular values below svd_eps sigma_1 changes the far field by a small multiple of
    svd_eps (bound 100 svd_eps of the largest far entry over three levels), and by nothing once no
    value falls below the cut."""
    O = oracle_mod
    o0, _ = _oracle(O, 600, 4, 6, getattr(O, kernel), kparam=(kp, 0, 0, 0))
    A0 = o0.dense_tilde()
    scale = np.abs(A0 - np.diag(np.diag(A0))).max()
    prev = None
    for se in (1e-5, 1e-7, 1e-9, 1e-11):
        o, _ = _oracle(O, 600, 4, 6, getattr(O, kernel), kparam=(kp, 0, 0, 0), svd_eps=se)
        err = np.abs(o.dense_tilde() - A0).max() / scale
        ranks = [o.svd_basis(k)[2] for k in (2, 3, 4)]
        assert err <= 100 * se, (se, err, ranks)
        if min(ranks) == 36:
            assert err <= 1e-13
        if prev is not None:
            assert sum(ranks) >= prev
        prev = sum(ranks)


def test_svd_compressed_solve_matches_dense_lu(oracle_mod):
    """Factor and solve with the truncated bases: the solution of A~ x = b (A~ the truncated FMM
    matrix, assembled densely) within C eps of its dense LU solution, C = 1e3 as in the uncompressed
    case."""
    O = oracle_mod
    N = 700
    o, pts = _oracle(O, N, 3, 5, O.K_LOG_REG, kparam=(0.001, 0, 0, 0), diag=1.0, eps=1e-10, tau_ref=1,
                     svd_eps=1e-8)
    rng = np.random.default_rng(5)
    b = rng.standard_normal(N)
    o.factor()
    x = o.solve(b)
    xd = np.linalg.solve(o.dense_tilde(), b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e3 * 1e-10
