"""The C-ABI library loads on the CPU host and exports every symbol include/ifmm.h declares."""
import ctypes
import os
import re

import pytest

from paper_1407_1572_gb300 import ifmm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "ifmm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ifmm_[A-Za-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol():
    lib = ifmm.load()
    declared = _declared()
    assert declared, "no declarations parsed"
    missing = [s for s in declared if not hasattr(lib, s)]
    assert not missing, missing
    assert sorted(ifmm.SYMBOLS) == declared


def test_default_params_and_struct_layout():
    p = ifmm.default_params()
    assert (p.dim, p.depth, p.cheb_p, p.precision, p.tau_ref) == (2, 3, 4, 0, 1)
    assert p.box[2] == 1.0 and p.eps == 1e-10 and p.refine_maxit == 100 and p.refine_restart == 60
    assert p.refine_inner == 1e-4 and p.leaf_max == 64 and p.tc_products == 0
    # host-side argument checks reject bad input without touching a device
    h = ctypes.c_void_p()
    lib = ifmm.load()
    import numpy as np
    pts = np.zeros((4, 2))
    bad = ifmm.default_params(depth=1)
    assert lib.ifmm_build(pts.ctypes.data_as(ctypes.c_void_p), 4, 0, ctypes.byref(bad), None, ctypes.byref(h)) == 1
    bad = ifmm.default_params(dim=4)
    assert lib.ifmm_build(pts.ctypes.data_as(ctypes.c_void_p), 4, 0, ctypes.byref(bad), None, ctypes.byref(h)) == 1
    assert p.svd_eps == 0.0 and p.z0 == 0.0
    pts[0, 0] = float("nan")
    ok = ifmm.default_params()
    assert lib.ifmm_build(pts.ctypes.data_as(ctypes.c_void_p), 4, 0, ctypes.byref(ok), None, ctypes.byref(h)) == 1
    assert lib.ifmm_factor(None) == 1
    assert lib.ifmm_solve(None, None, None, 1, 1) == 1


@pytest.mark.parametrize("change,kernel,n", [
    (dict(depth=11), 0, 4), (dict(cheb_p=0), 0, 4), (dict(cheb_p=9), 0, 4),
    (dict(depth=0, leaf_max=0), 0, 4), (dict(), 6, 4), (dict(), -1, 4),
    (dict(kparam=(0.0,)), 1, 4), (dict(kparam=(-1.0,)), 3, 4), (dict(kparam=(0.0,)), 5, 4),
    (dict(eps=-1e-6), 0, 4), (dict(diag=float("inf")), 0, 4), (dict(precision=3), 0, 4),
    (dict(tau_ref=3), 0, 4), (dict(r_cap=8), 0, 4), (dict(refine_restart=201), 0, 4),
    (dict(refine_restart=-1), 0, 4), (dict(tc_products=3), 0, 4), (dict(tc_products=-1), 0, 4), (dict(), 0, 0),
    (dict(svd_eps=-1e-3), 0, 4), (dict(svd_eps=1.0), 0, 4), (dict(dim=1), 0, 4),
    # octree limits: p^3 <= 64, an explicit depth <= 6, no tensor-core replay
    (dict(dim=3, cheb_p=5), 0, 4), (dict(dim=3, depth=0), 0, 4), (dict(dim=3, depth=7), 0, 4),
    (dict(dim=3, tc_products=1), 0, 4), (dict(dim=3, z0=float("nan")), 0, 4),
])
def test_build_rejects_each_out_of_range_argument_on_the_host(change, kernel, n):
    """Every range ifmm.h states for ifmm_build is checked before any device call: the call returns
    IFMM_ERR_INVALID_ARG and leaves the output handle NULL."""
    import numpy as np
    lib = ifmm.load()
    pts = np.full((max(n, 1), 3), 0.5)   # room for three coordinates per point
    prm = ifmm.default_params(**change)
    h = ctypes.c_void_p(1)
    st = lib.ifmm_build(pts.ctypes.data_as(ctypes.c_void_p), n, kernel, ctypes.byref(prm), None, ctypes.byref(h))
    assert st == ifmm.IFMM_ERR_INVALID_ARG
    assert not h.value


def test_no_cpu_fallback_without_a_device():
    """With valid arguments and no CUDA device the library fails with IFMM_ERR_CUDA and a message;
    nothing on the product path computes on the host instead."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    import numpy as np
    lib = ifmm.load()
    pts = np.random.default_rng(0).random((256, 2))
    prm = ifmm.default_params(depth=2)
    h = ctypes.c_void_p(1)
    st = lib.ifmm_build(pts.ctypes.data_as(ctypes.c_void_p), 256, 0, ctypes.byref(prm), None, ctypes.byref(h))
    assert st == ifmm.IFMM_ERR_CUDA and not h.value
    with pytest.raises(RuntimeError):   # the wrapper fails before the build (no CUDA stream)
        ifmm.IFMM(pts, ifmm.IFMM_K_INV_R, prm)


def test_compress_cluster_setting_is_checked_on_the_host():
    lib = ifmm.load()
    for bad in (0, 3, 32, -1):
        assert lib.ifmm_set_compress_cluster(bad) == 1
    for ok in (1, 2, 4, 8, 16):
        assert lib.ifmm_set_compress_cluster(ok) == 0
    with pytest.raises(ifmm.IFMMError):
        ifmm.ifmm_set_compress_cluster(5)
