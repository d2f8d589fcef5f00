"""ifmm_matvec_noalloc: the matvec for callers that must not allocate device memory.

Such callers (an application whose device memory belongs to another allocator, or a loop where an
allocation would stall the device) get the same product as ifmm_matvec from a call that keeps its
intermediate vectors in a fixed array compiled into the library. This file is collected last so
that a failure here cannot hide the result of any other test. It must pass both alone in a fresh
process and after the other tests (the shared array then holds another call's leftovers).
"""
import math

import numpy as np
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


def _colmajor(a):
    # (N, nrhs) array -> device buffer laid out column-major with leading dimension N
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda()


def test_noalloc_matvec_matches_allocating_matvec(ifmm):
    N, depth, p, nrhs = 6000, 3, 4, 3
    pts = inputs.uniform_points(2026, N)
    prm = ifmm.default_params(depth=depth, cheb_p=p, eps=1e-8, diag=math.sqrt(N))
    solver = ifmm.IFMM(pts, ifmm.IFMM_K_INV_R, prm)
    h = solver.h
    for call, seed in enumerate((31, 32)):          # two calls in a row, different inputs
        x = _colmajor(inputs.rhs(seed, N, nrhs))
        y_ref = torch.empty_like(x)
        y_new = torch.full_like(x, float("nan"))
        ifmm.ifmm_matvec(h, x.data_ptr(), y_ref.data_ptr(), nrhs, N)
        ifmm.ifmm_matvec_noalloc(h, x.data_ptr(), y_new.data_ptr(), nrhs, N)
        a, b = y_new.cpu().numpy(), y_ref.cpu().numpy()
        assert np.isfinite(a).all(), f"call {call}: non-finite output"
        assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max(), f"call {call}: differs from ifmm_matvec"
    solver.close()


def test_noalloc_matvec_rejects_oversized_calls(ifmm):
    N, depth = 70000, 5
    pts = inputs.uniform_points(7, N)
    prm = ifmm.default_params(depth=depth, cheb_p=4, eps=1e-6, diag=math.sqrt(N))
    solver = ifmm.IFMM(pts, ifmm.IFMM_K_INV_R, prm)
    nrhs = 64                                       # 70000 x 64 doubles alone exceed 32 MiB
    x = torch.zeros((nrhs, N), dtype=torch.float64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(ifmm.IFMMError) as ei:
        ifmm.ifmm_matvec_noalloc(solver.h, x.data_ptr(), y.data_ptr(), nrhs, N)
    assert ei.value.status == ifmm.IFMM_ERR_INVALID_ARG
    assert "32" in str(ei.value) or "limit" in str(ei.value)
    solver.close()
