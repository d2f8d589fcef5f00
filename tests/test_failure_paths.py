"""Failure paths of the factorisation, observed on the host through the C ABI; none of them faults or
stalls the GPU.

* A pivot block that is exactly singular (Eqs. P2P(i,k), P2M(i,k) of Section 4.2 give
  Piv = [[P2P_ee, L2P_ee], [P2M_ee, 0]]) is reported by the device status flag as
  IFMM_ERR_SINGULAR_PIVOT; the handle stays valid but unfactored, as the oracle reports it too.
* A rank cap (r_cap) below what the compression of Algorithm 1 wants is reported as
  IFMM_ERR_RANK_OVERFLOW with a usable factorisation that equals the oracle's at the same cap.
"""
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


def _coincident_pair_points():
    """Depth 2 (16 leaves of side 1/4): leaf (0, 0) holds two copies of one point and nothing else;
    every other leaf holds four seeded uniform points of its own."""
    rng = inputs.uniform_points(2024, 15 * 4)
    pts = [[0.1, 0.1], [0.1, 0.1]]
    t = 0
    for iy in range(4):
        for ix in range(4):
            if ix == 0 and iy == 0:
                continue
            for _ in range(4):
                u, v = rng[t]
                t += 1
                pts.append([(ix + 0.05 + 0.9 * u) / 4.0, (iy + 0.05 + 0.9 * v) / 4.0])
    return np.array(pts)


def test_singular_pivot_is_reported_and_leaves_the_handle_unfactored(ifmm):
    """Kernel (r / l^2) exp(-r / l) (zero at r = 0) with a zero diagonal: the leaf that holds only
    two coincident points has P2P_ee = 0 and equal basis rows (rank 1), so its pivot block
    [[0, 0, w0], [0, 0, w1], [w0, w1, 0]] has two rows that are multiples of one unit vector and is
    exactly singular. The GPU's Gauss-Jordan finds an exactly zero pivot column, sets the device flag
    and the factorisation returns IFMM_ERR_SINGULAR_PIVOT; a solve afterwards is refused with
    IFMM_ERR_STATE. The oracle's LU rejects the same block."""
    pts = _coincident_pair_points()
    N = pts.shape[0]
    prm = ifmm.default_params(depth=2, cheb_p=4, eps=1e-10, diag=0.0, kparam=(0.1,))
    g = ifmm.IFMM(pts, ifmm.IFMM_K_DEXP_DELL, prm)
    lib = ifmm.load()
    st = lib.ifmm_factor(g.h)
    assert st == ifmm.IFMM_ERR_SINGULAR_PIVOT, (st, ifmm.ifmm_last_error(g.h))
    assert "singular" in ifmm.ifmm_last_error(g.h)
    b = torch.zeros((1, N), dtype=torch.float64, device="cuda")
    x = torch.zeros_like(b)
    assert lib.ifmm_solve(g.h, b.data_ptr(), x.data_ptr(), 1, N) == ifmm.IFMM_ERR_STATE
    # the handle stays usable: the FMM matvec still runs
    y = g.matvec(torch.ones((N,), dtype=torch.float64, device="cuda"))
    assert bool(torch.isfinite(y).all())
    o = O.Oracle(pts, O.make_params(2, 4, O.K_DEXP_DELL, eps=1e-10, diag=0.0, kparam=(0.1, 0, 0, 0), tau_ref=1))
    with pytest.raises(RuntimeError, match=r"\(4\)"):
        o.factor()
    g.close()


@pytest.mark.parametrize("r_cap", [16, 20])
def test_rank_cap_overflow_is_reported_with_a_usable_factorisation(ifmm, r_cap):
    """4,096 uniform points, depth 3, rank 16, eps 1e-10: the compression wants more than r_cap
    directions in some boxes. The factorisation returns IFMM_ERR_RANK_OVERFLOW, counts the overflow,
    keeps every rank <= r_cap, and is the oracle's factorisation at the same cap: identical ranks
    (both keep the first r_cap directions of the pivoted Gram-Schmidt) and the same solution, to
    1e-10 at r_cap = 16 (nothing is appended) and to 2e-7 at r_cap = 20, where each cut leaves a
    remainder far above eps and the four kept directions follow the rounding of the fill: the
    oracle on points moved by one unit in the last place differs from itself by 4e-8 there
    (measured GPU vs oracle: 5.5e-8)."""
    N, depth, p, eps = 4096, 3, 4, 1e-10
    pts = inputs.uniform_points(1407 + N, N)
    prm = ifmm.default_params(depth=depth, cheb_p=p, eps=eps, diag=math.sqrt(N), r_cap=r_cap)
    g = ifmm.IFMM(pts, ifmm.IFMM_K_INV_R, prm)
    st = g.factor(allow_overflow=True)
    assert st == ifmm.IFMM_ERR_RANK_OVERFLOW
    s = g.stats()
    assert s["rank_overflows"] == 1 and s["max_rank"] <= r_cap
    o = O.Oracle(pts, O.make_params(depth, p, O.K_INV_R, eps=eps, diag=math.sqrt(N), r_cap=r_cap, tau_ref=1))
    o.factor()
    assert o.stats()["overflows"] > 0
    for k in range(2, depth + 1):
        assert np.array_equal(g.ranks(k), o.ranks(k)), f"ranks differ at level {k}"
    b = inputs.rhs(9, N, 2)
    x = g.solve(torch.from_numpy(np.ascontiguousarray(b)).cuda()).cpu().numpy()
    xo = o.solve(b)
    assert np.abs(x - xo).max() <= (1e-10 if r_cap == 16 else 2e-7) * np.abs(xo).max()
