"""The autotuner of the batched launches on the GPU, through the C ABI: tuning a batch of uneven
systems fills the table with one split per bucket, the systems it leaves factored solve to exactly
the untuned results (a split changes which block computes which output tile, never the arithmetic),
and the table saved to a file and loaded again gives the same results once more."""
import math

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


def test_tuned_splits_give_identical_results(ifmm, tmp_path):
    systems = [(inputs.uniform_points(41, 4000), 2), (inputs.gaussian_blobs(42, 6000), 3),
               (inputs.uniform_points(43, 16384), 1)]
    prm = [ifmm.default_params(depth=0, cheb_p=4, eps=1e-8, diag=math.sqrt(len(p)), tau_ref=1, precision=2)
           for p, _ in systems]
    hs = [ifmm.IFMM(p, 0, q) for (p, _), q in zip(systems, prm)]
    bs = [torch.from_numpy(inputs.rhs(50 + i, len(p), nr).T.copy()).cuda() for i, (p, nr) in enumerate(systems)]

    def solve_all():
        xs = []
        for g, b, (p, nr) in zip(hs, bs, systems):
            x = torch.empty_like(b)
            ifmm.ifmm_solve(g.h, b.data_ptr(), x.data_ptr(), nr, len(p))
            xs.append(x)
        torch.cuda.synchronize()
        return xs

    try:
        ifmm.ifmm_autotune_clear()
        ifmm.ifmm_factor_batch([g.h for g in hs])
        x0 = solve_all()
        size = ifmm.ifmm_autotune([g.h for g in hs])
        assert size > 0
        x1 = solve_all()
        for a, b in zip(x0, x1):
            assert torch.equal(a, b)
        path = tmp_path / "tune.txt"
        ifmm.ifmm_autotune_save(str(path))
        rows = [l.split() for l in path.read_text().splitlines() if l and not l.startswith("#")]
        assert len(rows) == size
        for k, df, lb, bb, z in rows:
            assert k in ("0", "1") and df == "1" and int(z) in (1, 2, 4, 8, 16)
        print("tuned table:", rows)
        ifmm.ifmm_autotune_clear()
        ifmm.ifmm_autotune_load(str(path))
        assert ifmm.ifmm_autotune_size() == size
        ifmm.ifmm_factor_batch([g.h for g in hs])
        x2 = solve_all()
        for a, b in zip(x0, x2):
            assert torch.equal(a, b)
    finally:
        ifmm.ifmm_autotune_clear()
        for g in hs:
            g.close()
