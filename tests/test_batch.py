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


def test_mixed_mode_blob_systems_reach_tolerance(ifmm):
    """Gaussian-blob systems of the batched workload (clustered points: more ill-conditioned pivot
    blocks than uniform clouds) solved in the mixed mode through the batch API reach the
    manufactured solutions within 1e-6."""
    sy = [s for i, s in enumerate(inputs.batch_systems(count=256)) if i in (128, 160, 192, 224, 250, 255)]
    streams = [torch.cuda.Stream() for _ in sy]
    hs, xs_l, bs_l, xo_l = [], [], [], []
    for s, st in zip(sy, streams):
        n = s["points"].shape[0]
        prm = ifmm.default_params(depth=0, cheb_p=4, eps=1e-6, diag=math.sqrt(n), tau_ref=1,
                                  precision=ifmm.IFMM_MIXED_SOLVE, refine_tol=1e-7, refine_maxit=120)
        g = ifmm.IFMM(s["points"], 0, prm, st)
        xs = torch.from_numpy(inputs.rhs(s["seed"], n, s["nrhs"]).T.copy()).cuda()
        b = torch.empty_like(xs)
        ifmm.ifmm_matvec(g.h, xs.data_ptr(), b.data_ptr(), s["nrhs"], n)
        hs.append(g); xs_l.append(xs); bs_l.append(b); xo_l.append(torch.empty_like(xs))
    torch.cuda.synchronize()
    ifmm.ifmm_factor_batch([g.h for g in hs], workers=6, allow_overflow=True)
    ifmm.ifmm_solve_batch([g.h for g in hs], [b.data_ptr() for b in bs_l], [x.data_ptr() for x in xo_l],
                          [s["nrhs"] for s in sy], [s["points"].shape[0] for s in sy], workers=6)
    torch.cuda.synchronize()
    for x, xs in zip(xo_l, xs_l):
        assert float(((x - xs).norm(dim=1) / xs.norm(dim=1)).max()) <= 1e-6
    for g in hs:
        g.close()
