"""Planted mistakes: each of nine plausible errors, compiled into a copy of the oracle
(-DORACLE_PLANT=k), makes at least one pin of tests/test_oracle_pins.py fail, while the same pins
pass on the unplanted build. This checks the pins themselves: a pin set that a dropped term, a
wrong sign or index, or a wrong threshold slips through would not pin the oracle."""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "ifmm_oracle.cpp")
PINS = os.path.join(ROOT, "tests", "test_oracle_pins.py")

PLANTS = {
    1: "row M2L_e of Algorithm 1 updated with the wrong sign at the neighbours' columns",
    2: "the P2L redirect (P2L_pq = M2L_pq P2M_qq) perturbed by a relative 1e-6",
    3: "one child's L2L missing from the parent's L2P (Eq. particles_multipoles)",
    4: "the new column y_e formed with +I instead of -I at z_e",
    5: "the forward replay's update perturbed by a relative 1e-6",
    6: "the children's x and y offsets swapped in the solve's level transition",
    7: "the compression threshold taken relative to the fill instead of eps * s_A",
    8: "no re-orthogonalisation of a Gram-Schmidt candidate",
    9: "one direction too few kept by the compression",
}


def _compile(k, out_dir):
    lib = os.path.join(out_dir, f"liboracle_plant{k}.so")
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", f"-DORACLE_PLANT={k}",
                           "-o", lib, SRC])
    return lib


def _run_pins(lib):
    env = dict(os.environ, ORACLE_LIB_OVERRIDE=lib, OMP_NUM_THREADS="2")
    res = subprocess.run([sys.executable, "-m", "pytest", PINS, "-x", "-q", "-p", "no:cacheprovider"], cwd=ROOT,
                         env=env, capture_output=True, text=True)
    return res.returncode, res.stdout[-2000:]


def test_each_planted_mistake_fails_a_pin(tmp_path):
    if subprocess.run(["g++", "--version"], capture_output=True).returncode != 0:
        pytest.skip("no C++ compiler")
    ks = [0] + sorted(PLANTS)
    with cf.ThreadPoolExecutor(max_workers=len(ks)) as ex:
        libs = dict(zip(ks, ex.map(lambda k: _compile(k, str(tmp_path)), ks)))
        runs = dict(zip(ks, ex.map(lambda k: _run_pins(libs[k]), ks)))
    rc0, out0 = runs[0]
    assert rc0 == 0, "the unplanted oracle must pass its pins:\n" + out0
    caught = {k: runs[k][0] != 0 for k in PLANTS}
    missed = [PLANTS[k] for k, c in caught.items() if not c]
    assert not missed, f"pins passed despite: {missed}"
