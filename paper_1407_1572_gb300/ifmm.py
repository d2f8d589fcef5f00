"""Thin Python binding of the C ABI in include/ifmm.h (argument marshalling only).

Every step of build, factor, solve and matvec runs in the CUDA kernels of libifmm_gb300.so.
PyTorch provides device memory and streams. If the library cannot be loaded the import fails:
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

IFMM_OK, IFMM_ERR_INVALID_ARG, IFMM_ERR_CUDA, IFMM_ERR_OOM = 0, 1, 2, 3
IFMM_ERR_SINGULAR_PIVOT, IFMM_ERR_RANK_OVERFLOW, IFMM_ERR_NOCONV = 4, 5, 6
IFMM_ERR_TIMEOUT, IFMM_ERR_STATE = 7, 8
IFMM_K_INV_R, IFMM_K_EXP, IFMM_K_DEXP_DELL = 0, 1, 2
IFMM_K_LOG_REG, IFMM_K_INV_REG, IFMM_K_R2LOG_REG = 3, 4, 5   # Section 5 benchmark kernels
IFMM_FP64, IFMM_MIXED, IFMM_MIXED_SOLVE = 0, 1, 2
_NAMES = {0: "IFMM_OK", 1: "IFMM_ERR_INVALID_ARG", 2: "IFMM_ERR_CUDA", 3: "IFMM_ERR_OOM",
          4: "IFMM_ERR_SINGULAR_PIVOT", 5: "IFMM_ERR_RANK_OVERFLOW", 6: "IFMM_ERR_NOCONV",
          7: "IFMM_ERR_TIMEOUT", 8: "IFMM_ERR_STATE"}


class ifmm_params(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("depth", ctypes.c_int), ("cheb_p", ctypes.c_int),
                ("r_cap", ctypes.c_int), ("eps", ctypes.c_double), ("diag", ctypes.c_double),
                ("kparam", ctypes.c_double * 4), ("box", ctypes.c_double * 3),
                ("precision", ctypes.c_int), ("tau_ref", ctypes.c_int),
                ("refine_tol", ctypes.c_double), ("refine_maxit", ctypes.c_int),
                ("refine_restart", ctypes.c_int),
                ("refine_inner", ctypes.c_double),
                ("leaf_max", ctypes.c_int), ("tc_products", ctypes.c_int), ("svd_eps", ctypes.c_double), ("z0", ctypes.c_double)]


class ifmm_stats(ctypes.Structure):
    _fields_ = [("n_points", ctypes.c_int64), ("depth", ctypes.c_int), ("max_rank", ctypes.c_int),
                ("rank_overflows", ctypes.c_int), ("refine_iters", ctypes.c_int),
                ("t_build_ms", ctypes.c_double), ("t_factor_ms", ctypes.c_double),
                ("t_solve_ms", ctypes.c_double), ("factor_flops", ctypes.c_double),
                ("schur_flops", ctypes.c_double), ("schur_bytes", ctypes.c_double),
                ("kernel_ms", ctypes.c_double * 5), ("kernel_launches", ctypes.c_int * 5),
                ("kernel_flops", ctypes.c_double * 5), ("level_ms", ctypes.c_double * 16),
                ("last_update", ctypes.c_double), ("last_residual", ctypes.c_double),
                ("device_bytes", ctypes.c_int64), ("launches_factor", ctypes.c_int64),
                ("launches_solve", ctypes.c_int64), ("compress_proj_flops", ctypes.c_double),
                ("svd_ranks", ctypes.c_int * 16), ("compress_reorth_flops", ctypes.c_double)]


FACTOR_KERNELS = ("k_pivot", "k_panel", "k_schur", "k_compress", "k_redirect")


class IFMMError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

# every symbol include/ifmm.h declares
SYMBOLS = ["ifmm_default_params", "ifmm_auto_depth", "ifmm_build", "ifmm_factor", "ifmm_factor_batch",
           "ifmm_solve", "ifmm_solve_T", "ifmm_solve_batch", "ifmm_solve_host",
           "ifmm_matvec", "ifmm_matvec_noalloc", "ifmm_tc_dgemm", "ifmm_get_ranks", "ifmm_get_stats",
           "ifmm_last_error", "ifmm_destroy", "ifmm_autotune", "ifmm_autotune_save", "ifmm_autotune_load",
           "ifmm_autotune_clear", "ifmm_autotune_size", "ifmm_set_compress_cluster"]


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libifmm_gb300.so (building it in-tree first if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise OSError(f"{path} is missing; run paper_1407_1572_gb300.build.build()")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, i64, ip = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
    lib.ifmm_default_params.argtypes = [ctypes.POINTER(ifmm_params)]
    lib.ifmm_default_params.restype = None
    lib.ifmm_build.argtypes = [vp, i64, ip, ctypes.POINTER(ifmm_params), vp, ctypes.POINTER(vp)]
    lib.ifmm_build.restype = ip
    lib.ifmm_factor.argtypes = [vp]
    lib.ifmm_factor.restype = ip
    for name in ("ifmm_solve", "ifmm_solve_T", "ifmm_solve_host", "ifmm_matvec", "ifmm_matvec_noalloc"):
        getattr(lib, name).argtypes = [vp, vp, vp, ip, i64]
        getattr(lib, name).restype = ip
    lib.ifmm_tc_dgemm.argtypes = [vp, i64, vp, i64, vp, i64, ip, ip, ip, vp]
    lib.ifmm_tc_dgemm.restype = ip
    lib.ifmm_get_ranks.argtypes = [vp, ip, vp]
    lib.ifmm_get_ranks.restype = ip
    lib.ifmm_get_stats.argtypes = [vp, ctypes.POINTER(ifmm_stats)]
    lib.ifmm_get_stats.restype = ip
    lib.ifmm_last_error.argtypes = [vp]
    lib.ifmm_last_error.restype = ctypes.c_char_p
    lib.ifmm_destroy.argtypes = [vp]
    lib.ifmm_destroy.restype = None
    lib.ifmm_auto_depth.argtypes = [vp, i64, vp, ip]
    lib.ifmm_auto_depth.restype = ip
    lib.ifmm_factor_batch.argtypes = [ctypes.POINTER(vp), ip, ip, ctypes.POINTER(ip)]
    lib.ifmm_factor_batch.restype = ip
    lib.ifmm_solve_batch.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                     ctypes.POINTER(ip), ctypes.POINTER(i64), ip, ctypes.POINTER(ip)]
    lib.ifmm_solve_batch.restype = ip
    lib.ifmm_autotune.argtypes = [ctypes.POINTER(vp), ip, ip]
    lib.ifmm_autotune.restype = ip
    for name in ("ifmm_autotune_save", "ifmm_autotune_load"):
        getattr(lib, name).argtypes = [ctypes.c_char_p]
        getattr(lib, name).restype = ip
    lib.ifmm_autotune_clear.argtypes = []
    lib.ifmm_autotune_clear.restype = None
    lib.ifmm_autotune_size.argtypes = []
    lib.ifmm_autotune_size.restype = ip
    lib.ifmm_set_compress_cluster.argtypes = [ip]
    lib.ifmm_set_compress_cluster.restype = ip
    _lib = lib
    return lib


def default_params(**kw) -> ifmm_params:
    p = ifmm_params()
    load().ifmm_default_params(ctypes.byref(p))
    for k, v in kw.items():
        if k in ("kparam", "box"):
            arr = getattr(p, k)
            for i, x in enumerate(v):
                arr[i] = float(x)
        else:
            setattr(p, k, v)
    return p


def _check(h, status: int, allow=()):
    if status != IFMM_OK and status not in allow:
        msg = load().ifmm_last_error(h).decode() if h else ""
        raise IFMMError(status, msg)
    return status


# ---- C-ABI names ---------------------------------------------------------------------------

def ifmm_build(points: np.ndarray, kernel: int, params: ifmm_params, stream: int = 0):
    """points: N x dim (params.dim = 2 or 3)."""
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, params.dim)
    h = ctypes.c_void_p()
    st = load().ifmm_build(pts.ctypes.data_as(ctypes.c_void_p), pts.shape[0], kernel, ctypes.byref(params),
                           ctypes.c_void_p(stream), ctypes.byref(h))
    _check(None, st)
    return h


def ifmm_auto_depth(points: np.ndarray, leaf_max: int = 64, box=None) -> int:
    pts = np.ascontiguousarray(points, dtype=np.float64).reshape(-1, 2)
    bx = None if box is None else np.ascontiguousarray(box, dtype=np.float64)
    return load().ifmm_auto_depth(pts.ctypes.data_as(ctypes.c_void_p), pts.shape[0],
                                  None if bx is None else bx.ctypes.data_as(ctypes.c_void_p), leaf_max)


def ifmm_factor_batch(handles, workers: int = 0, allow_overflow: bool = False):
    """Factor the systems of `handles` concurrently; returns the per-system statuses."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    st = (ctypes.c_int * n)()
    load().ifmm_factor_batch(hs, n, workers, st)
    out = list(st)
    bad = [i for i, v in enumerate(out) if v not in ((IFMM_OK, IFMM_ERR_RANK_OVERFLOW) if allow_overflow else (IFMM_OK,))]
    if bad:
        raise IFMMError(out[bad[0]], f"system {bad[0]}: " + load().ifmm_last_error(handles[bad[0]]).decode())
    return out


def ifmm_autotune(handles, workers: int = 0) -> int:
    """Tune the panel / Schur launch splits on these systems (see include/ifmm.h); returns the size of
    the process-wide table. The systems are left factored."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    _check(None, load().ifmm_autotune(hs, n, workers), allow=(IFMM_ERR_RANK_OVERFLOW,))
    return load().ifmm_autotune_size()


def ifmm_autotune_save(path: str) -> None:
    _check(None, load().ifmm_autotune_save(os.fsencode(path)))


def ifmm_autotune_load(path: str) -> None:
    _check(None, load().ifmm_autotune_load(os.fsencode(path)))


def ifmm_autotune_clear() -> None:
    load().ifmm_autotune_clear()


def ifmm_autotune_size() -> int:
    return load().ifmm_autotune_size()


def ifmm_set_compress_cluster(max_blocks: int) -> None:
    """Largest cluster one compression may be spread over (1, 2, 4, 8 or 16; 1 turns clusters off)."""
    _check(None, load().ifmm_set_compress_cluster(int(max_blocks)))


def ifmm_solve_batch(handles, b_ptrs, x_ptrs, nrhs, lds, workers: int = 0, allow_noconv: bool = False):
    """Solve the factored systems of `handles` concurrently (device pointers, column-major)."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    bp = (ctypes.c_void_p * n)(*b_ptrs)
    xp = (ctypes.c_void_p * n)(*x_ptrs)
    nr = (ctypes.c_int * n)(*nrhs)
    ld = (ctypes.c_int64 * n)(*lds)
    st = (ctypes.c_int * n)()
    load().ifmm_solve_batch(hs, n, bp, xp, nr, ld, workers, st)
    out = list(st)
    bad = [i for i, v in enumerate(out) if v not in ((IFMM_OK, IFMM_ERR_NOCONV) if allow_noconv else (IFMM_OK,))]
    if bad:
        raise IFMMError(out[bad[0]], f"system {bad[0]}: " + load().ifmm_last_error(handles[bad[0]]).decode())
    return out


def ifmm_factor(h, allow_overflow: bool = False) -> int:
    return _check(h, load().ifmm_factor(h), allow=(IFMM_ERR_RANK_OVERFLOW,) if allow_overflow else ())


def ifmm_solve(h, b_ptr: int, x_ptr: int, nrhs: int, ld: int, allow_noconv: bool = False) -> int:
    return _check(h, load().ifmm_solve(h, ctypes.c_void_p(b_ptr), ctypes.c_void_p(x_ptr), nrhs, ld),
                  allow=(IFMM_ERR_NOCONV,) if allow_noconv else ())


def ifmm_solve_T(h, b_ptr: int, x_ptr: int, nrhs: int, ld: int, allow_noconv: bool = False) -> int:
    return _check(h, load().ifmm_solve_T(h, ctypes.c_void_p(b_ptr), ctypes.c_void_p(x_ptr), nrhs, ld),
                  allow=(IFMM_ERR_NOCONV,) if allow_noconv else ())


def ifmm_solve_host(h, b: np.ndarray, x: np.ndarray, nrhs: int, ld: int, allow_noconv: bool = False) -> int:
    return _check(h, load().ifmm_solve_host(h, b.ctypes.data_as(ctypes.c_void_p), x.ctypes.data_as(ctypes.c_void_p),
                                            nrhs, ld), allow=(IFMM_ERR_NOCONV,) if allow_noconv else ())


def ifmm_matvec(h, x_ptr: int, y_ptr: int, nrhs: int, ld: int) -> int:
    return _check(h, load().ifmm_matvec(h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), nrhs, ld))


def ifmm_matvec_noalloc(h, x_ptr: int, y_ptr: int, nrhs: int, ld: int) -> int:
    """ifmm_matvec without device allocation (fixed 32 MiB scratch compiled into the library)."""
    return _check(h, load().ifmm_matvec_noalloc(h, ctypes.c_void_p(x_ptr), ctypes.c_void_p(y_ptr), nrhs, ld))


def ifmm_tc_dgemm(a_ptr: int, lda: int, b_ptr: int, ldb: int, c_ptr: int, ldc: int, M: int, N: int, K: int,
                  stream: int = 0) -> int:
    """C = A B (row-major FP64 device arrays) on the tensor cores in FP64 accuracy."""
    return _check(None, load().ifmm_tc_dgemm(a_ptr, lda, b_ptr, ldb, c_ptr, ldc, M, N, K, stream))


def ifmm_get_ranks(h, level: int, dim: int = 2) -> np.ndarray:
    out = np.zeros(1 << (dim * level), dtype=np.int32)
    _check(h, load().ifmm_get_ranks(h, level, out.ctypes.data_as(ctypes.c_void_p)))
    return out


def ifmm_get_stats(h) -> dict:
    s = ifmm_stats()
    _check(h, load().ifmm_get_stats(h, ctypes.byref(s)))
    out = {}
    for name, _ in ifmm_stats._fields_:
        v = getattr(s, name)
        out[name] = list(v) if name in ("kernel_ms", "kernel_launches", "kernel_flops", "level_ms", "svd_ranks") else v
    return out


def ifmm_last_error(h) -> str:
    return load().ifmm_last_error(h).decode()


def ifmm_destroy(h) -> None:
    if h:
        load().ifmm_destroy(h)


# ---- convenience wrapper over torch tensors ---------------------------------------------------

class IFMM:
    """One problem: build at construction, then factor() and solve(b) / matvec(x).

    Vectors are torch tensors on the device, shape (N,) or (N, nrhs), float64, in the caller's
    point order; they are passed to the C ABI as column-major arrays with leading dimension N.
    """

    def __init__(self, points: np.ndarray, kernel: int = IFMM_K_INV_R, params: ifmm_params | None = None,
                 stream=None):
        import torch
        self._torch = torch
        self.params = params if params is not None else default_params()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.N = int(np.asarray(points).reshape(-1, self.params.dim).shape[0])
        self.h = ifmm_build(points, kernel, self.params, self.stream.cuda_stream)

    def close(self):
        if getattr(self, "h", None):
            ifmm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def factor(self, allow_overflow: bool = False) -> int:
        return ifmm_factor(self.h, allow_overflow)

    def _colmajor(self, v):
        torch = self._torch
        if v.dim() == 1:
            v = v.unsqueeze(1)
        if v.shape[0] != self.N:
            raise ValueError("first dimension must be N")
        return v.to(dtype=torch.float64).t().contiguous()   # (nrhs, N): column-major N x nrhs

    def solve(self, b, allow_noconv: bool = False):
        bt = self._colmajor(b)
        xt = self._torch.empty_like(bt)
        ifmm_solve(self.h, bt.data_ptr(), xt.data_ptr(), bt.shape[0], self.N, allow_noconv)
        x = xt.t()
        return x[:, 0] if b.dim() == 1 else x

    def solve_T(self, b, allow_noconv: bool = False):
        bt = self._colmajor(b)
        xt = self._torch.empty_like(bt)
        ifmm_solve_T(self.h, bt.data_ptr(), xt.data_ptr(), bt.shape[0], self.N, allow_noconv)
        x = xt.t()
        return x[:, 0] if b.dim() == 1 else x

    def matvec(self, x):
        xt = self._colmajor(x)
        yt = self._torch.empty_like(xt)
        ifmm_matvec(self.h, xt.data_ptr(), yt.data_ptr(), xt.shape[0], self.N)
        y = yt.t()
        return y[:, 0] if x.dim() == 1 else y

    def solve_host(self, b: np.ndarray, allow_noconv: bool = False) -> np.ndarray:
        b2 = np.asfortranarray(np.asarray(b, dtype=np.float64).reshape(self.N, -1))
        x = np.zeros_like(b2, order="F")
        ifmm_solve_host(self.h, b2, x, b2.shape[1], self.N, allow_noconv)
        return x.reshape(np.asarray(b).shape)

    def ranks(self, level: int) -> np.ndarray:
        return ifmm_get_ranks(self.h, level, self.params.dim)

    def stats(self) -> dict:
        return ifmm_get_stats(self.h)
