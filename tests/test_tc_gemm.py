"""The tensor-core FP64 product (ifmm_tc_dgemm, the Schur-update product of Algorithm 1) through the C
ABI, against exact arithmetic.

* Exactly representable inputs (integers below 2^20, so every entry has at most 21 significant
  bits and every exact product and sum fits in FP64): the result equals the exact integer product
  bit for bit -- the check that the digit split, the tensor-memory accumulators and the integer
  combination lose nothing.
* FP64 inputs with rows and columns scaled over 2^+-30: every sampled entry within 2^-48 |A| |B|
  of the exact value (a sum of exact rational products; eight 7-bit digits per entry leave about
  2^-52 in a bit-exact emulation), and the whole result within 2^-48 |A| |B| + 2 K u |A| |B| of
  the FP64 product.
* Ragged and degenerate shapes: M, N not multiples of the 128 x 32 tile, K below one MMA step
  (16), K across several read-backs of the accumulators (128), a zero row and a zero column.
"""
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ifmm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_1572_gb300 import ifmm as m
    m.load()
    return m


def _tc(ifmm, A, B):
    A = np.ascontiguousarray(A, dtype=np.float64)
    B = np.ascontiguousarray(B, dtype=np.float64)
    M, K = A.shape
    N = B.shape[1]
    a, b = torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda()
    c = torch.full((M, N), float("nan"), dtype=torch.float64, device="cuda")
    ifmm.ifmm_tc_dgemm(a.data_ptr(), K, b.data_ptr(), N, c.data_ptr(), N, M, N, K)
    return c.cpu().numpy()


@pytest.mark.parametrize("M,N,K", [(128, 32, 32), (200, 70, 64), (37, 5, 9), (130, 33, 300), (1, 1, 1),
                                   (256, 96, 512)])
def test_integer_inputs_are_exact(ifmm, M, N, K):
    rng = np.random.default_rng(M * 1000 + N * 10 + K)
    A = rng.integers(-(1 << 20), 1 << 20, size=(M, K))
    B = rng.integers(-(1 << 20), 1 << 20, size=(K, N))
    exact = A @ B                                   # int64: |sum| < 512 * 2^40 = 2^49
    C = _tc(ifmm, A.astype(np.float64), B.astype(np.float64))
    assert np.array_equal(C, exact.astype(np.float64))


@pytest.mark.parametrize("M,N,K", [(150, 40, 100), (64, 64, 64), (33, 97, 257)])
def test_fp64_inputs_within_the_split_bound(ifmm, M, N, K):
    rng = np.random.default_rng(7 + M + N + K)
    A = rng.standard_normal((M, K)) * np.exp2(rng.integers(-30, 30, size=(M, 1)))
    B = rng.standard_normal((K, N)) * np.exp2(rng.integers(-30, 30, size=(1, N)))
    A[M // 2, :] = 0.0                               # a zero row and a zero column
    B[:, N // 3] = 0.0
    C = _tc(ifmm, A, B)
    absAB = np.abs(A) @ np.abs(B)
    u = 2.0 ** -53
    assert np.all(np.abs(C - A @ B) <= (2.0 ** -48 + 2 * K * u) * absAB)
    assert np.all(C[M // 2, :] == 0.0) and np.all(C[:, N // 3] == 0.0)
    # sampled entries against the exact sum of exact products
    for t in range(40):
        i, j = int(rng.integers(0, M)), int(rng.integers(0, N))
        ex = sum((Fraction(float(A[i, k])) * Fraction(float(B[k, j])) for k in range(K)), Fraction(0))
        err = abs(Fraction(float(C[i, j])) - ex)
        assert err <= Fraction(2.0 ** -48) * Fraction(float(absAB[i, j])), (i, j, float(err), absAB[i, j])


def test_wide_dynamic_range(ifmm):
    """Entries from 1e-150 to 1e+150 across rows and columns (each row and column has its own power
    of two scale), products far from over- or underflow."""
    rng = np.random.default_rng(3)
    M, N, K = 64, 40, 80
    A = rng.standard_normal((M, K)) * (10.0 ** rng.uniform(-150, 150, size=(M, 1)))
    B = rng.standard_normal((K, N)) * (10.0 ** rng.uniform(-100, 100, size=(1, N)))
    C = _tc(ifmm, A, B)
    absAB = np.abs(A) @ np.abs(B)
    assert np.all(np.abs(C - A @ B) <= (2.0 ** -48 + 2 * K * 2.0 ** -53) * absAB)
