"""The octree (d = 3, Section 4.2's extension of the method to three dimensions) on the GPU, through
the C ABI, against the CPU oracle on the same seeded points: the FMM matvec element by element,
then factor and solve (identical ranks, solution element-wise), in FP64 and in the mixed solve.

Workloads: points uniform in the unit cube, 1/r + sqrt(N) I (the 3D Laplace kernel) and exp(-r/l),
Chebyshev 3 x 3 x 3 (rank 27) or 4 x 4 x 4 (rank 64), one or two elimination levels for the solves
(the oracle's 3D elimination takes minutes beyond that) and three for the matvec; ragged leaves
(N not a multiple of the leaf count) and a Gaussian-blob cloud with empty leaves.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1407_1572_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu

_OK = {0: O.K_INV_R, 1: O.K_EXP}


@pytest.fixture(scope="module")
def ifmm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_1572_gb300 import ifmm as m
    m.load()
    return m


def _pts(seed, N, blobs=False):
    if not blobs:
        return inputs.uniform(seed, 3 * N).reshape(N, 3)
    rng = np.random.default_rng(seed)
    centres = 0.15 + 0.7 * rng.random((6, 3))
    p = centres[rng.integers(0, 6, N)] + 0.06 * rng.standard_normal((N, 3))
    return np.clip(p, 0.0, 1.0)


def _pair(ifmm, pts, depth, p, eps, kernel=0, kp=0.0, precision=0, refine_tol=0.0):
    N = pts.shape[0]
    d = math.sqrt(N)
    prm = ifmm.default_params(dim=3, depth=depth, cheb_p=p, eps=eps, diag=d, kparam=(kp,), tau_ref=1,
                              precision=precision, refine_tol=refine_tol, refine_maxit=40)
    g = ifmm.IFMM(pts, kernel, prm)
    o = O.Oracle(pts, O.make_params(depth, p, _OK[kernel], eps=eps, diag=d, kparam=(kp, 0, 0, 0), tau_ref=1, dim=3))
    return g, o


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _maxrel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("N,depth,p,kernel", [(3001, 2, 3, 0), (12000, 3, 3, 0), (9000, 3, 4, 1), (30011, 4, 3, 0)])
def test_matvec_3d_matches_oracle(ifmm, N, depth, p, kernel):
    pts = _pts(300 + N, N)
    g, o = _pair(ifmm, pts, depth, p, 1e-8, kernel, 0.25)
    x = inputs.rhs(5, N, 2)
    d = _maxrel(g.matvec(_t(x)).cpu().numpy(), o.matvec(x))
    print(f"3D matvec N={N} depth={depth} p={p}: GPU vs oracle {d:.2e}")
    assert d <= 1e-12


@pytest.mark.parametrize("N,depth,p,eps,bar,blobs", [
    (3001, 2, 3, 1e-10, 1e-10, False),    # one elimination level, ragged leaves
    (8000, 3, 3, 1e-6, 1e-8, False),      # two levels, 512 leaves of ~16 points
    (6000, 3, 4, 1e-6, 1e-8, False),      # rank 64
    (6000, 3, 3, 1e-6, 1e-8, True),       # Gaussian blobs: empty and crowded leaves
])
def test_fp64_factor_solve_3d_matches_oracle(ifmm, N, depth, p, eps, bar, blobs):
    """Identical box ranks at every level and the solution element-wise within `bar` of the
    oracle's (relative to its largest element), as in 2D."""
    pts = _pts(700 + N, N, blobs)
    g, o = _pair(ifmm, pts, depth, p, eps)
    g.factor()
    o.factor()
    for k in range(2, depth + 1):
        gr, orr = g.ranks(k), o.ranks(k)
        nd = int((gr != orr).sum())
        print(f"level {k}: {nd} of {gr.size} ranks differ (max rank {orr.max()})")
        assert np.array_equal(gr, orr), f"ranks differ at level {k}"
    b = inputs.rhs(9, N, 2)
    x = g.solve(_t(b)).cpu().numpy()
    xo = o.solve(b)
    d = _maxrel(x, xo)
    print(f"3D N={N} p={p} eps={eps:g}: GPU vs oracle {d:.2e}")
    assert d <= bar


def test_uncompressed_3d_solve_is_the_dense_solve(ifmm):
    """eps = 0: the GPU's elimination reproduces A~^{-1} b (A~ assembled densely by the oracle's
    nested operators, solved by LU) to rounding."""
    N = 2500
    pts = _pts(41, N)
    g, o = _pair(ifmm, pts, 2, 3, 0.0)
    g.factor()
    b = inputs.rhs(12, N, 1)
    x = g.solve(_t(b)).cpu().numpy()
    xd = np.linalg.solve(o.dense_tilde(), b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-11


def test_mixed_solve_3d_reaches_the_fp64_solution(ifmm):
    """IFMM_MIXED_SOLVE (FP64 elimination, double-float solve phase) with refinement to 1e-10 on the
    octree: the solution within 1e-9 of the oracle's FP64 factor + solve refined the same way by
    dense iterations (here: the dense solve of the oracle's A~)."""
    N = 8000
    pts = _pts(77, N)
    g, o = _pair(ifmm, pts, 3, 3, 1e-6, precision=2, refine_tol=1e-10)
    g.factor()
    b = inputs.rhs(13, N, 2)
    x = g.solve(_t(b)).cpu().numpy()
    o.factor()
    xo = o.solve(b)
    # refine the oracle's solution with its own matvec and solve (classical refinement, FP64)
    for _ in range(30):
        r = b - o.matvec(xo)
        xo = xo + o.solve(r)
        if np.linalg.norm(o.solve(b - o.matvec(xo))) <= 1e-12 * np.linalg.norm(xo):
            break
    d = _maxrel(x, xo)
    print(f"3D mixed solve vs refined oracle: {d:.2e}, iterations {g.stats()['refine_iters']}")
    assert d <= 1e-9
