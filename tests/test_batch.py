"""Batched systems (uneven N, uniform and Gaussian-blob point clouds, automatic depth, empty leaves):
the batch API gives every system exactly the result it gets alone, and a blob cloud with empty
leaves matches the oracle."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_1407_1572_gb300 import inputs  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ifmm():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1407_1572_gb300 import ifmm as m
    m.load()
    return m


def _prm(ifmm, n, **kw):
    return ifmm.default_params(depth=0, cheb_p=4, eps=1e-8, diag=math.sqrt(n), tau_ref=1, **kw)


def test_batch_equals_individual_solves(ifmm):
    systems = [(inputs.uniform_points(21, 2000), 1), (inputs.gaussian_blobs(22, 3000), 3),
               (inputs.uniform_points(23, 9000), 2), (inputs.gaussian_blobs(24, 12000), 5),
               (inputs.uniform_points(25, 5000), 4), (inputs.gaussian_blobs(26, 6000), 1)]
    streams = [torch.cuda.Stream() for _ in systems]
    batch = [ifmm.IFMM(pts, 0, _prm(ifmm, len(pts)), st) for (pts, _), st in zip(systems, streams)]
    ifmm.ifmm_factor_batch([g.h for g in batch], workers=4)
    bs = [torch.from_numpy(inputs.rhs(30 + i, len(pts), nr).T.copy()).cuda() for i, (pts, nr) in enumerate(systems)]
    xs = [torch.empty_like(b) for b in bs]
    torch.cuda.synchronize()
    ifmm.ifmm_solve_batch([g.h for g in batch], [b.data_ptr() for b in bs], [x.data_ptr() for x in xs],
                          [nr for _, nr in systems], [len(p) for p, _ in systems], workers=4)
    torch.cuda.synchronize()
    for i, ((pts, nr), g) in enumerate(zip(systems, batch)):
        depth = g.stats()["depth"]
        assert depth == ifmm.ifmm_auto_depth(pts, 64)
        single = ifmm.IFMM(pts, 0, _prm(ifmm, len(pts)))
        single.factor()
        for k in range(2, depth + 1):
            assert np.array_equal(single.ranks(k), g.ranks(k))
        x1 = torch.empty_like(bs[i])
        ifmm.ifmm_solve(single.h, bs[i].data_ptr(), x1.data_ptr(), nr, len(pts))
        torch.cuda.synchronize()
        assert torch.equal(xs[i], x1), f"system {i} differs from its single solve"
        single.close()
    for g in batch:
        g.close()


def test_blob_cloud_with_empty_leaves_matches_oracle(ifmm):
    N = 3000
    pts = inputs.gaussian_blobs(31, N)
    depth = ifmm.ifmm_auto_depth(pts, 64)
    g = ifmm.IFMM(pts, 0, ifmm.default_params(depth=depth, cheb_p=4, eps=1e-10, diag=math.sqrt(N), tau_ref=1))
    g.factor()
    o = O.Oracle(pts, O.make_params(depth, 4, O.K_INV_R, eps=1e-10, diag=math.sqrt(N), tau_ref=1))
    o.factor()
    assert (o.leaf_counts() == 0).sum() > 0, "the cloud should leave empty leaves"
    for k in range(2, depth + 1):
        assert np.array_equal(g.ranks(k), o.ranks(k)), f"ranks differ at level {k}"
    b = inputs.rhs(32, N, 2)
    x = g.solve(torch.from_numpy(np.ascontiguousarray(b)).cuda()).cpu().numpy()
    xo = o.solve(b)
    rel = float(np.linalg.norm(x - xo) / np.linalg.norm(xo))
    print(f"blob cloud N={N} depth {depth}: GPU vs oracle {rel:.2e}")
    assert rel <= 1e-10
