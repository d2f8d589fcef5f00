"""Adjoint gradients through the IFMM solve for A(l, sigma2) = exp(-r/l) + sigma2 I, loss
||x - x*||^2 with x = A~^{-1} b: dL/db, dL/dl and dL/dsigma2 against the dense reference (the
oracle's assembled A~ and dA~/dl, dense solves) and against central differences of the loss."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1407_1572_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def adj():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_1572_gb300 import adjoint, ifmm
    ifmm.load()
    return adjoint


def _loss_and_grads(adj, pts, b, xs, ell, sig2, **prm):
    bt = torch.tensor(b, dtype=torch.float64, device="cuda", requires_grad=True)
    ell_t = torch.tensor(ell, dtype=torch.float64, device="cuda", requires_grad=True)
    sig_t = torch.tensor(sig2, dtype=torch.float64, device="cuda", requires_grad=True)
    xs_t = torch.tensor(xs, dtype=torch.float64, device="cuda")
    x = adj.solve_exp(pts, bt, ell_t, sig_t, **prm)
    loss = ((x - xs_t) ** 2).sum()
    loss.backward()
    return float(loss.detach()), bt.grad.cpu().numpy(), float(ell_t.grad), float(sig_t.grad)


def _loss(adj, pts, b, xs, ell, sig2, **prm):
    sysm = adj.ExpKernelSystem(pts, ell, sig2, **prm)
    x = sysm.solve(torch.tensor(b, dtype=torch.float64, device="cuda")).cpu().numpy()
    sysm.close()
    return float(((x - xs) ** 2).sum())


def test_gradients_match_dense_reference_and_differences(adj):
    N, depth, p, eps = 4096, 3, 6, 1e-8
    ell, sig2 = 0.1, 1e-2
    pts = inputs.uniform_points(1410, N)
    b = inputs.rhs(1412, N, 2)
    xs = inputs.rhs(1413, N, 2)
    prm = dict(depth=depth, cheb_p=p, eps=eps, tau_ref=1, refine_tol=1e-12, refine_maxit=80)
    L, g_b, g_ell, g_sig = _loss_and_grads(adj, pts, b, xs, ell, sig2, **prm)
    # dense reference: the FMM matrices the library factors and multiplies
    A = O.Oracle(pts, O.make_params(depth, p, O.K_EXP, eps=eps, diag=1.0 + sig2, kparam=(ell, 0, 0, 0))).dense_tilde()
    D = O.Oracle(pts, O.make_params(depth, p, O.K_DEXP_DELL, eps=eps, diag=0.0, kparam=(ell, 0, 0, 0))).dense_tilde()
    xd = np.linalg.solve(A, b)
    lam = np.linalg.solve(A.T, 2.0 * (xd - xs))
    assert L == pytest.approx(float(((xd - xs) ** 2).sum()), rel=1e-9)
    assert np.linalg.norm(g_b - lam) <= 1e-8 * np.linalg.norm(lam)
    assert g_sig == pytest.approx(-float((lam * xd).sum()), rel=1e-8)
    assert g_ell == pytest.approx(-float((lam * (D @ xd)).sum()), rel=1e-8)
    # central differences of the loss computed by the library
    for name, h in (("ell", 1e-4 * ell), ("sig2", 1e-4 * sig2)):
        if name == "ell":
            fd = (_loss(adj, pts, b, xs, ell + h, sig2, **prm) - _loss(adj, pts, b, xs, ell - h, sig2, **prm)) / (2 * h)
            assert g_ell == pytest.approx(fd, rel=1e-5)
        else:
            fd = (_loss(adj, pts, b, xs, ell, sig2 + h, **prm) - _loss(adj, pts, b, xs, ell, sig2 - h, **prm)) / (2 * h)
            assert g_sig == pytest.approx(fd, rel=1e-5)


def test_gradients_at_65536_points_match_differences(adj):
    """N = 65,536 uniform points, rank 36, eps 1e-8, l = 0.1, sigma2 = 1e-2 (the adjoint workload):
    dL/dl and dL/dsigma2 against central differences of the library's own loss."""
    N, depth, p, eps = 65536, 5, 6, 1e-8
    ell, sig2 = 0.1, 1e-2
    pts = inputs.uniform_points(1411, N)
    b = inputs.rhs(1414, N, 1)
    xs = inputs.rhs(1415, N, 1)
    prm = dict(depth=depth, cheb_p=p, eps=eps, tau_ref=1, refine_tol=1e-12, refine_maxit=80)
    _, _, g_ell, g_sig = _loss_and_grads(adj, pts, b, xs, ell, sig2, **prm)
    h = 1e-4 * ell
    fd = (_loss(adj, pts, b, xs, ell + h, sig2, **prm) - _loss(adj, pts, b, xs, ell - h, sig2, **prm)) / (2 * h)
    assert g_ell == pytest.approx(fd, rel=1e-5)
    h = 1e-4 * sig2
    fd = (_loss(adj, pts, b, xs, ell, sig2 + h, **prm) - _loss(adj, pts, b, xs, ell, sig2 - h, **prm)) / (2 * h)
    assert g_sig == pytest.approx(fd, rel=1e-5)
    assert math.isfinite(g_ell) and math.isfinite(g_sig)
