"""The compression of Algorithm 1 (Section 4.2) spread over thread-block clusters at the upper levels
(each block a slice of the stacked fill's columns, the pivot column chosen over the cluster) gives
the same ranks, bases and solutions bit for bit as one block per compression: quadtree in the mixed
solve and in FP64, and an octree (27 colours, few boxes per colour at every level)."""
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
    yield m
    m.ifmm_set_compress_cluster(16)


def _run(ifmm, pts, prm, nrhs, seed):
    g = ifmm.IFMM(pts, 0, prm)
    g.factor()
    depth = g.stats()["depth"]
    ranks = [g.ranks(k).copy() for k in range(2, depth + 1)]
    b = torch.from_numpy(inputs.rhs(seed, pts.shape[0], nrhs).T.copy()).cuda()
    x = torch.empty_like(b)
    ifmm.ifmm_solve(g.h, b.data_ptr(), x.data_ptr(), nrhs, pts.shape[0])
    torch.cuda.synchronize()
    g.close()
    return ranks, x.cpu()


@pytest.mark.parametrize("dim,N,depth,p,precision", [
    (2, 65536, 5, 4, "mixed_solve"),
    (2, 16384, 4, 6, "fp64"),
    (3, 12000, 2, 3, "fp64"),
])
def test_clustered_compression_is_bitwise_the_single_block_one(ifmm, dim, N, depth, p, precision):
    if dim == 2:
        pts = inputs.uniform_points(1407 + N, N)
    else:
        pts = inputs.uniform(1407 + N, 3 * N).reshape(N, 3)
    prec = {"mixed_solve": ifmm.IFMM_MIXED_SOLVE, "fp64": ifmm.IFMM_FP64}[precision]
    prm = ifmm.default_params(dim=dim, depth=depth, cheb_p=p, eps=1e-6, diag=math.sqrt(N), tau_ref=1,
                              precision=prec, refine_tol=0.0, refine_maxit=0)
    out = {}
    try:
        for c in (1, 4, 16):
            ifmm.ifmm_set_compress_cluster(c)
            out[c] = _run(ifmm, pts, prm, 4, 31 + N)
    finally:
        ifmm.ifmm_set_compress_cluster(16)
    r1, x1 = out[1]
    for c in (4, 16):
        rc, xc = out[c]
        assert len(r1) == len(rc)
        for k, (a, b) in enumerate(zip(r1, rc)):
            assert np.array_equal(a, b), f"cluster {c}: ranks differ at level {k + 2}"
        assert torch.equal(x1, xc), f"cluster {c}: solutions differ: max {float((x1 - xc).abs().max()):.3e}"
