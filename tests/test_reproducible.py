"""The refinement's reductions over N (Krylov dot products, column norms, residual norms) are summed
in a fixed order (per-block partials added in block order), so a GMRES-refined solve gives the same
bits every time it is repeated on the same factorisation, and a second factorisation of the same
system gives the same bits again; likewise the classical refinement."""
import math

import pytest

torch = pytest.importorskip("torch")

from paper_1407_1572_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ifmm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_1572_gb300 import ifmm as m
    m.load()
    return m


@pytest.mark.parametrize("precision,restart", [("mixed_solve", 60), ("fp64", 60), ("fp64", 0)])
def test_refined_solves_repeat_bit_for_bit(ifmm, precision, restart):
    N, nrhs = 16384, 4
    prec = {"mixed_solve": ifmm.IFMM_MIXED_SOLVE, "fp64": ifmm.IFMM_FP64}[precision]
    pts = inputs.uniform_points(3141, N)
    prm = ifmm.default_params(depth=4, cheb_p=4, eps=1e-6, diag=math.sqrt(N), tau_ref=1, precision=prec,
                              refine_tol=1e-9, refine_maxit=60, refine_restart=restart)
    b = torch.from_numpy(inputs.rhs(3142, N, nrhs).T.copy()).cuda()
    xs, its = [], []
    for _ in range(2):
        g = ifmm.IFMM(pts, 0, prm)
        g.factor()
        for _ in range(2):
            x = torch.empty_like(b)
            ifmm.ifmm_solve(g.h, b.data_ptr(), x.data_ptr(), nrhs, N, allow_noconv=True)
            torch.cuda.synchronize()
            xs.append(x.cpu())
            its.append(g.stats()["refine_iters"])
        g.close()
    assert min(its) >= 2, its
    for k in range(1, len(xs)):
        assert its[k] == its[0]
        assert torch.equal(xs[k], xs[0]), f"solve {k} differs: max {float((xs[k] - xs[0]).abs().max()):.3e}"
