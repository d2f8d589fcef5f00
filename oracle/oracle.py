"""ctypes binding of the CPU oracle (ifmm_oracle.cpp).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the package smoke check and by the bench's
CPU-baseline leg. The product library never imports it.

The oracle is a plain FP64 CPU restatement of the Inverse Fast Multipole Method
(Ambikasaran & Darve, arXiv:1407.1572): tree and lists (Section 4.2, Table "table_cluster"),
Chebyshev operators (Section 5), the extended sparse system (Section 4.1), Algorithm 1
(elimination with fill compression) and Algorithm 2 (back substitution).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ifmm_oracle.cpp")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "libifmm_oracle.so")
_lock = threading.Lock()
_lib = None

K_INV_R, K_EXP, K_DEXP_DELL, K_POLY = 0, 1, 2, 3
K_LOG_REG, K_INV_REG, K_R2LOG_REG = 4, 5, 6   # the numerical benchmarks of Section 5
K_R2 = 7                                       # |x - y|^2 (separable rank 4 in 2D: an SVD pin)


def compile_oracle(force: bool = False) -> str:
    """Compile the oracle shared library in-tree (plain g++, OpenMP)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ifmm_oracle.h")))
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
        tmp = _LIB + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared",
                               "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [("depth", ctypes.c_int), ("cheb_p", ctypes.c_int), ("kernel", ctypes.c_int),
                ("r_cap", ctypes.c_int), ("eps", ctypes.c_double), ("diag", ctypes.c_double),
                ("kparam", ctypes.c_double * 4), ("box", ctypes.c_double * 3),
                ("order", ctypes.c_int), ("threads", ctypes.c_int), ("tau_ref", ctypes.c_int),
                ("svd_eps", ctypes.c_double), ("dim", ctypes.c_int), ("z0", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = os.environ.get("ORACLE_LIB_OVERRIDE") or compile_oracle()
            lib = ctypes.CDLL(path)
            vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p
            lib.oracle_build.restype = vp
            lib.oracle_build.argtypes = [dp, i64, ctypes.POINTER(Params)]
            lib.oracle_destroy.argtypes = [vp]
            for name in ("oracle_factor",):
                getattr(lib, name).argtypes = [vp]
            for name in ("oracle_solve", "oracle_matvec", "oracle_extended_solve"):
                getattr(lib, name).argtypes = [vp, dp, dp, ctypes.c_int]
            for name in ("oracle_dense_tilde", "oracle_dense_tilde_direct", "oracle_dense_exact"):
                getattr(lib, name).argtypes = [vp, dp]
            lib.oracle_dense_lu_solve.argtypes = [dp, i64, dp, dp, ctypes.c_int]
            lib.oracle_ranks.argtypes = [vp, ctypes.c_int, dp]
            lib.oracle_initial_ranks.argtypes = [vp, ctypes.c_int, dp]
            lib.oracle_leaf_counts.argtypes = [vp, dp]
            lib.oracle_perm.argtypes = [vp, dp]
            lib.oracle_lists.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp, dp, dp, dp]
            lib.oracle_order.argtypes = [vp, ctypes.c_int, dp]
            lib.oracle_stats.argtypes = [vp, dp, ctypes.c_int]
            lib.oracle_cheb_nodes.argtypes = [ctypes.c_int, dp]
            lib.oracle_lagrange.argtypes = [ctypes.c_int, ctypes.c_double, dp]
            lib.oracle_kernel_eval.argtypes = [ctypes.POINTER(Params), dp, dp, dp]
            lib.oracle_kernel_matrix.argtypes = [ctypes.POINTER(Params), dp, i64, dp, i64, dp]
            lib.oracle_svd_basis.argtypes = [vp, ctypes.c_int, dp, dp]
            lib.oracle_augment_basis.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_int, dp, dp]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def make_params(depth, cheb_p, kernel=K_INV_R, eps=1e-10, diag=1.0, r_cap=0, kparam=(0, 0, 0, 0),
                box=(0.0, 0.0, 1.0), order=0, threads=0, tau_ref=0, svd_eps=0.0, dim=2, z0=0.0) -> Params:
    """box = (x0, y0, side); in 3D (dim = 3) the root cube also starts at z0."""
    p = Params()
    p.depth, p.cheb_p, p.kernel, p.r_cap = depth, cheb_p, kernel, r_cap
    p.eps, p.diag = eps, diag
    for i in range(4):
        p.kparam[i] = float(kparam[i]) if i < len(kparam) else 0.0
    for i in range(3):
        p.box[i] = float(box[i])
    p.order, p.threads, p.tau_ref = order, threads, tau_ref
    p.svd_eps = svd_eps
    p.dim, p.z0 = dim, z0
    return p


def cheb_nodes(p: int) -> np.ndarray:
    t = np.zeros(p)
    _load().oracle_cheb_nodes(p, _ptr(t))
    return t


def lagrange(p: int, t: float) -> np.ndarray:
    out = np.zeros(p)
    _load().oracle_lagrange(p, float(t), _ptr(out))
    return out


def kernel_eval(params: Params, a, b) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.zeros(1)
    _load().oracle_kernel_eval(ctypes.byref(params), _ptr(a), _ptr(b), _ptr(out))
    return float(out[0])


def kernel_matrix(params: Params, P, Q) -> np.ndarray:
    """K(P_i, Q_j) for point sets P (m x dim) and Q (n x dim): the kernel alone, no diagonal term."""
    d = params.dim if params.dim else 2
    P = np.ascontiguousarray(P, dtype=np.float64).reshape(-1, d)
    Q = np.ascontiguousarray(Q, dtype=np.float64).reshape(-1, d)
    out = np.zeros((P.shape[0], Q.shape[0]))
    _load().oracle_kernel_matrix(ctypes.byref(params), _ptr(P), P.shape[0], _ptr(Q), Q.shape[0], _ptr(out))
    return out


def augment_basis(W: np.ndarray, S: np.ndarray, eps: float, ref: float = 0.0, cap: int = 0):
    """Reading R2's compression step alone: returns (extended basis, appended count, overflow).
    W: n x r with orthonormal columns (r may be 0), S: n x m fill; threshold eps * ref (ref > 0) or
    eps * the largest column norm of S."""
    S = np.ascontiguousarray(S, dtype=np.float64)
    n, m = S.shape
    W = np.ascontiguousarray(np.asarray(W, dtype=np.float64).reshape(n, -1))
    r = W.shape[1]
    out = np.zeros(n * n)
    ov = np.zeros(1, dtype=np.int32)
    add = _load().oracle_augment_basis(_ptr(W) if r else None, n, r, _ptr(S), m, float(eps), float(ref), int(cap),
                                       _ptr(out), _ptr(ov))
    if add < 0:
        raise ValueError("oracle_augment_basis rejected its arguments")
    return out[: n * (r + add)].reshape(n, r + add), int(add), bool(ov[0])


def dense_lu_solve(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    A = np.ascontiguousarray(A, dtype=np.float64)
    b2 = b.reshape(b.shape[0], -1)
    bc = np.asfortranarray(b2, dtype=np.float64)
    x = np.zeros_like(bc, order="F")
    rc = _load().oracle_dense_lu_solve(_ptr(A), A.shape[0], _ptr(bc), _ptr(x), bc.shape[1])
    if rc:
        raise RuntimeError(f"oracle dense LU failed ({rc})")
    return x.reshape(b.shape)


class Oracle:
    """One IFMM problem on the CPU oracle: build at construction, then factor / solve."""

    def __init__(self, points: np.ndarray, params: Params):
        self._lib = _load()
        self.dim = params.dim if params.dim else 2
        pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, self.dim)
        self.N = pts.shape[0]
        self.params = params
        self.depth = params.depth
        self._h = self._lib.oracle_build(_ptr(pts), self.N, ctypes.byref(params))
        if not self._h:
            raise ValueError("oracle_build rejected its arguments")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_destroy(h)
            self._h = None

    def _vec_call(self, fn, b: np.ndarray) -> np.ndarray:
        b2 = b.reshape(self.N, -1)
        bc = np.asfortranarray(b2, dtype=np.float64)
        out = np.zeros_like(bc, order="F")
        rc = fn(self._h, _ptr(bc), _ptr(out), bc.shape[1])
        if rc:
            raise RuntimeError(f"oracle call failed ({rc})")
        return out.reshape(b.shape)

    def factor(self) -> None:
        rc = self._lib.oracle_factor(self._h)
        if rc:
            raise RuntimeError(f"oracle_factor failed ({rc})")

    def solve(self, b: np.ndarray) -> np.ndarray:
        return self._vec_call(self._lib.oracle_solve, b)

    def matvec(self, x: np.ndarray) -> np.ndarray:
        return self._vec_call(self._lib.oracle_matvec, x)

    def extended_solve(self, b: np.ndarray) -> np.ndarray:
        return self._vec_call(self._lib.oracle_extended_solve, b)

    def _dense(self, fn) -> np.ndarray:
        A = np.zeros((self.N, self.N))
        rc = fn(self._h, _ptr(A))
        if rc:
            raise RuntimeError(f"oracle dense assembly failed ({rc})")
        return A

    def dense_tilde(self) -> np.ndarray:
        return self._dense(self._lib.oracle_dense_tilde)

    def dense_tilde_direct(self) -> np.ndarray:
        return self._dense(self._lib.oracle_dense_tilde_direct)

    def dense_exact(self) -> np.ndarray:
        return self._dense(self._lib.oracle_dense_exact)

    def num_boxes(self, level: int) -> int:
        """Boxes of a level: 2^(dim level)."""
        return 1 << (self.dim * level)

    def ranks(self, level: int) -> np.ndarray:
        out = np.zeros(self.num_boxes(level), dtype=np.int32)
        rc = self._lib.oracle_ranks(self._h, level, _ptr(out))
        if rc:
            raise RuntimeError("oracle_ranks: not factored")
        return out

    def initial_ranks(self, level: int) -> np.ndarray:
        out = np.zeros(self.num_boxes(level), dtype=np.int32)
        self._lib.oracle_initial_ranks(self._h, level, _ptr(out))
        return out

    def svd_basis(self, level: int):
        """(U, sigma, r): the SVD of the level's M2L kernel matrices (Section 5's compression of the
        Chebyshev interpolation) and the number of singular values the handle's svd_eps keeps."""
        r0 = self.params.cheb_p ** 2
        U = np.zeros((r0, r0))
        sg = np.zeros(r0)
        r = self._lib.oracle_svd_basis(self._h, level, _ptr(U), _ptr(sg))
        if r < 0:
            raise ValueError("oracle_svd_basis: bad level")
        return U, sg, int(r)

    def leaf_counts(self) -> np.ndarray:
        out = np.zeros(self.num_boxes(self.depth), dtype=np.int32)
        self._lib.oracle_leaf_counts(self._h, _ptr(out))
        return out

    def perm(self) -> np.ndarray:
        out = np.zeros(self.N, dtype=np.int64)
        self._lib.oracle_perm(self._h, _ptr(out))
        return out

    def lists(self, level: int, box: int):
        nb = np.zeros(self.num_boxes(level), dtype=np.int32)
        it = np.zeros(self.num_boxes(level), dtype=np.int32)
        nn = np.zeros(1, dtype=np.int32)
        ni = np.zeros(1, dtype=np.int32)
        self._lib.oracle_lists(self._h, level, box, _ptr(nb), _ptr(nn), _ptr(it), _ptr(ni))
        return nb[: nn[0]].copy(), it[: ni[0]].copy()

    def order(self, level: int) -> np.ndarray:
        out = np.zeros(self.num_boxes(level), dtype=np.int32)
        self._lib.oracle_order(self._h, level, _ptr(out))
        return out

    def stats(self) -> dict:
        out = np.zeros(9)
        self._lib.oracle_stats(self._h, _ptr(out), 9)
        keys = ["flops", "bytes", "compressions", "overflows", "max_rank", "eliminations",
                "directions_added", "factor_seconds", "scale_A"]
        return dict(zip(keys, out.tolist()))
