"""The C-ABI library loads on the CPU host and exports every symbol include/ifmm.h declares."""
import ctypes
import os
import re

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
    assert p.refine_inner == 1e-4 and p.leaf_max == 64
    # host-side argument checks reject bad input without touching a device
    h = ctypes.c_void_p()
    lib = ifmm.load()
    import numpy as np
    pts = np.zeros((4, 2))
    bad = ifmm.default_params(depth=1)
    assert lib.ifmm_build(pts.ctypes.data_as(ctypes.c_void_p), 4, 0, ctypes.byref(bad), None, ctypes.byref(h)) == 1
    bad = ifmm.default_params(dim=3)
    assert lib.ifmm_build(pts.ctypes.data_as(ctypes.c_void_p), 4, 0, ctypes.byref(bad), None, ctypes.byref(h)) == 1
    pts[0, 0] = float("nan")
    ok = ifmm.default_params()
    assert lib.ifmm_build(pts.ctypes.data_as(ctypes.c_void_p), 4, 0, ctypes.byref(ok), None, ctypes.byref(h)) == 1
    assert lib.ifmm_factor(None) == 1
    assert lib.ifmm_solve(None, None, None, 1, 1) == 1
