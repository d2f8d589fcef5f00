"""Gradients through the IFMM solve (adjoint method) for A(theta) = exp(-|x - y| / l) + sigma2 I.

For x = A~(theta)^{-1} b and a loss L(x) with g = dL/dx, the adjoint lambda = A~^{-T} g gives

    dL/db = lambda,   dL/d sigma2 = -lambda^T x,   dL/dl = -lambda^T (dA~/dl) x.

lambda comes from `ifmm_solve_T` through the same factors as the forward solve. dA~/dl x is the FMM
matvec of the kernel (r / l^2) exp(-r / l) with a zero diagonal: the tree, the Chebyshev nodes and
the orthonormal bases of the FMM do not depend on l, so differentiating the FMM matrix A~(l) gives
the FMM matrix of the differentiated kernel (Table "table_FMM_operators"; the far-field blocks are
U K(xbar_i, ybar_j) V^T with U, V and the nodes fixed). The gradient is therefore the gradient of
the computed solution, to the accuracy of the refined solves.

The solves and the matvecs run in the library's CUDA kernels; the two inner products that turn
lambda into dL/dl and dL/dsigma2 are plain torch reductions on the device tensors.
"""
from __future__ import annotations

import numpy as np

from . import ifmm as _ifmm


class ExpKernelSystem:
    """IFMM of A(l, sigma2) = exp(-r / l) + sigma2 I on fixed points, factored once, plus the FMM
    matvec of dA/dl on the same tree. `params` are keyword arguments of `ifmm.default_params`
    (depth, cheb_p, eps, precision, refine_tol, ...); kparam and diag are set here."""

    def __init__(self, points: np.ndarray, ell: float, sigma2: float, stream=None, **params):
        if not (ell > 0.0):
            raise ValueError("the length scale must be positive")
        self.ell, self.sigma2 = float(ell), float(sigma2)
        prm = _ifmm.default_params(**params)
        prm.kparam[0] = self.ell
        prm.diag = 1.0 + self.sigma2          # K(x, x) = 1 plus the shift
        self.A = _ifmm.IFMM(points, _ifmm.IFMM_K_EXP, prm, stream)
        self.A.factor()
        dprm = _ifmm.default_params(**params)
        dprm.kparam[0] = self.ell
        dprm.diag = 0.0                       # d(sigma2 I)/dl = 0 and dK/dl vanishes at r = 0
        self.dA = _ifmm.IFMM(points, _ifmm.IFMM_K_DEXP_DELL, dprm, stream)

    def solve(self, b):
        return self.A.solve(b)

    def solve_T(self, g):
        return self.A.solve_T(g)

    def dA_dl_matvec(self, x):
        return self.dA.matvec(x)

    def close(self):
        for h in (getattr(self, "A", None), getattr(self, "dA", None)):
            if h is not None:
                h.close()


def _function():
    import torch

    class IFMMSolveExp(torch.autograd.Function):
        """x = A(l, sigma2)^{-1} b with the adjoint gradients for b, l and sigma2."""

        @staticmethod
        def forward(ctx, b, ell, sigma2, system):
            x = system.solve(b)
            ctx.system = system
            ctx.save_for_backward(x)
            return x

        @staticmethod
        def backward(ctx, g):
            (x,) = ctx.saved_tensors
            system = ctx.system
            lam = system.solve_T(g.contiguous())
            g_b = lam if ctx.needs_input_grad[0] else None
            g_ell = g_sig = None
            if ctx.needs_input_grad[1]:
                g_ell = -(lam * system.dA_dl_matvec(x)).sum().reshape(())
            if ctx.needs_input_grad[2]:
                g_sig = -(lam * x).sum().reshape(())
            return g_b, g_ell, g_sig, None

    return IFMMSolveExp


_FN = None


def solve_exp(points: np.ndarray, b, ell, sigma2, system: ExpKernelSystem | None = None, **params):
    """Differentiable x = A(l, sigma2)^{-1} b. `b` is a float64 CUDA tensor (N,) or (N, nrhs); `ell`
    and `sigma2` are 0-dimensional tensors (they may require grad). A `system` built for the same
    points and parameter values may be passed to reuse its factorisation; otherwise one is built
    (and released when the returned tensor's graph is freed)."""
    global _FN
    if _FN is None:
        _FN = _function()
    ell_v = float(ell.detach()) if hasattr(ell, "detach") else float(ell)
    sig_v = float(sigma2.detach()) if hasattr(sigma2, "detach") else float(sigma2)
    if system is None:
        system = ExpKernelSystem(points, ell_v, sig_v, **params)
    elif system.ell != ell_v or system.sigma2 != sig_v:
        raise ValueError("the system was built for other parameter values")
    return _FN.apply(b, ell, sigma2, system)
