"""Edge cases of the CUDA path through the C ABI: leading dimensions larger than N (device and host
buffers), columns solved alone against a block of right-hand sides, the largest number of
right-hand sides, tiny systems whose tree is mostly empty, and points on the upper edges of the
root box (clamped into the last box)."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1407_1572_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ifmm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_1572_gb300 import ifmm as m
    m.load()
    return m


def _solver(ifmm, pts, depth=3, p=4, eps=1e-10):
    n = pts.shape[0]
    g = ifmm.IFMM(pts, ifmm.IFMM_K_INV_R, ifmm.default_params(depth=depth, cheb_p=p, eps=eps, diag=math.sqrt(n)))
    g.factor()
    return g


def test_leading_dimension_larger_than_n(ifmm):
    n, nrhs, pad = 3001, 3, 7
    g = _solver(ifmm, inputs.uniform_points(41, n))
    b = inputs.rhs(42, n, nrhs)
    bt = torch.from_numpy(np.ascontiguousarray(b.T)).cuda()              # ld = n
    x_tight = torch.empty_like(bt)
    ifmm.ifmm_solve(g.h, bt.data_ptr(), x_tight.data_ptr(), nrhs, n)
    bp = torch.full((nrhs, n + pad), float("nan"), dtype=torch.float64, device="cuda")
    bp[:, :n] = bt
    xp = torch.full_like(bp, 7.0)
    ifmm.ifmm_solve(g.h, bp.data_ptr(), xp.data_ptr(), nrhs, n + pad)   # ld = n + pad, NaN padding unread
    torch.cuda.synchronize()
    assert torch.equal(xp[:, :n], x_tight)
    assert bool((xp[:, n:] == 7.0).all()), "the padding of x must not be written"
    y_tight = torch.empty_like(bt)
    ifmm.ifmm_matvec(g.h, bt.data_ptr(), y_tight.data_ptr(), nrhs, n)
    yp = torch.full_like(bp, 7.0)
    ifmm.ifmm_matvec(g.h, bp.data_ptr(), yp.data_ptr(), nrhs, n + pad)
    torch.cuda.synchronize()
    assert torch.equal(yp[:, :n], y_tight)
    # host buffers: one copy per column when ld > N, one block copy when ld = N
    bh = np.full((nrhs, n + pad), np.nan)
    bh[:, :n] = b.T
    xh = np.full_like(bh, 7.0)
    ifmm.ifmm_solve_host(g.h, bh, xh, nrhs, n + pad)
    assert np.array_equal(xh[:, :n], x_tight.cpu().numpy())
    assert bool((xh[:, n:] == 7.0).all()), "the padding of the host x must not be written"
    xt = np.zeros((nrhs, n))
    ifmm.ifmm_solve_host(g.h, np.ascontiguousarray(b.T), xt, nrhs, n)
    assert np.array_equal(xt, x_tight.cpu().numpy())
    g.close()


def test_columns_alone_equal_the_block_solve(ifmm):
    n, nrhs = 4096, 5
    g = _solver(ifmm, inputs.uniform_points(43, n), eps=1e-8)
    b = torch.from_numpy(np.ascontiguousarray(inputs.rhs(44, n, nrhs).T)).cuda()
    xb = torch.empty_like(b)
    ifmm.ifmm_solve(g.h, b.data_ptr(), xb.data_ptr(), nrhs, n)
    for j in range(nrhs):
        xj = torch.empty((1, n), dtype=torch.float64, device="cuda")
        ifmm.ifmm_solve(g.h, b[j].contiguous().data_ptr(), xj.data_ptr(), 1, n)
        torch.cuda.synchronize()
        assert torch.equal(xj[0], xb[j]), f"column {j}"
    g.close()


def test_largest_number_of_right_hand_sides(ifmm):
    n, nrhs = 1024, 1024
    pts = inputs.uniform_points(45, n)
    g = _solver(ifmm, pts, depth=2, p=3, eps=1e-10)
    b = inputs.rhs(46, n, nrhs)
    x = g.solve(torch.from_numpy(np.ascontiguousarray(b)).cuda()).cpu().numpy()
    o = O.Oracle(pts, O.make_params(2, 3, O.K_INV_R, eps=1e-10, diag=math.sqrt(n), tau_ref=1))
    o.factor()
    cols = [0, 511, 1023]
    xo = o.solve(np.ascontiguousarray(b[:, cols]))
    assert np.linalg.norm(x[:, cols] - xo) <= 1e-10 * np.linalg.norm(xo)
    with pytest.raises(ifmm.IFMMError):
        bt = torch.zeros((nrhs + 1, n), dtype=torch.float64, device="cuda")
        ifmm.ifmm_solve(g.h, bt.data_ptr(), bt.data_ptr(), nrhs + 1, n)
    g.close()


@pytest.mark.parametrize("n,depth", [(5, 2), (37, 3), (200, 4)])
def test_tiny_systems_on_mostly_empty_trees(ifmm, n, depth):
    pts = inputs.uniform_points(47 + n, n)
    g = _solver(ifmm, pts, depth=depth, p=3, eps=1e-12)
    o = O.Oracle(pts, O.make_params(depth, 3, O.K_INV_R, eps=1e-12, diag=math.sqrt(n), tau_ref=1))
    o.factor()
    for k in range(2, depth + 1):
        assert np.array_equal(g.ranks(k), o.ranks(k))
    b = inputs.rhs(48, n, 2)
    x = g.solve(torch.from_numpy(np.ascontiguousarray(b)).cuda()).cpu().numpy()
    A = o.dense_tilde()
    assert np.linalg.norm(x - np.linalg.solve(A, b)) <= 1e-9 * np.linalg.norm(np.linalg.solve(A, b))
    g.close()


def test_points_on_the_upper_box_edges(ifmm):
    """Points at coordinate 1 fall into the last box of their row or column (exact check of the
    leaf counts) and give identical ranks; the solution gate is 1e-9 (measured 2.4e-10): with 81
    points moved onto two edges this set is less well conditioned than the uniform ones, and the
    GPU and the oracle differ by FP64 rounding order."""
    n = 2000
    pts = inputs.uniform_points(49, n)
    pts[:40, 0] = 1.0          # right edge
    pts[40:80, 1] = 1.0        # top edge
    pts[80] = (1.0, 1.0)       # corner
    pts[81] = (0.0, 0.0)
    g = _solver(ifmm, pts, depth=3, p=4, eps=1e-10)
    o = O.Oracle(pts, O.make_params(3, 4, O.K_INV_R, eps=1e-10, diag=math.sqrt(n), tau_ref=1))
    o.factor()
    assert np.array_equal(np.sort(o.leaf_counts()), np.sort(np.bincount(
        np.minimum((pts[:, 1] * 8).astype(int), 7) * 8 + np.minimum((pts[:, 0] * 8).astype(int), 7), minlength=64)))
    for k in range(2, 4):
        assert np.array_equal(g.ranks(k), o.ranks(k))
    b = inputs.rhs(50, n, 1)
    x = g.solve(torch.from_numpy(np.ascontiguousarray(b)).cuda()).cpu().numpy()
    xo = o.solve(b)
    assert np.linalg.norm(x - xo) <= 1e-9 * np.linalg.norm(xo)
    g.close()
