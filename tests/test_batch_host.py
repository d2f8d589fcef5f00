"""Host logic of the batched workload (no GPU): the automatic tree depth through the C ABI against a
brute-force count, and the seeded generators of uniform / Gaussian-blob systems."""
import numpy as np

from paper_1407_1572_gb300 import ifmm, inputs


def _brute_depth(pts, leaf_max, box=(0.0, 0.0, 1.0)):
    x0, y0, L = box
    for depth in range(2, 11):
        side = 2 ** depth
        ux = np.clip((pts[:, 0] - x0) / L, 0.0, 1.0)
        uy = np.clip((pts[:, 1] - y0) / L, 0.0, 1.0)
        ix = np.minimum(np.floor(ux * side).astype(int), side - 1)
        iy = np.minimum(np.floor(uy * side).astype(int), side - 1)
        if np.bincount(iy * side + ix, minlength=side * side).max() <= leaf_max:
            return depth
    return 10


def test_auto_depth_matches_brute_force():
    cases = [(inputs.uniform_points(5, 4000), 64, None), (inputs.gaussian_blobs(6, 5000), 64, None),
             (inputs.uniform_points(7, 700, lo=-1.0, side=2.0), 16, (-1.0, -1.0, 2.0)),
             (inputs.gaussian_blobs(8, 20000), 64, None)]
    for pts, lm, box in cases:
        want = _brute_depth(pts, lm, box if box is not None else (0.0, 0.0, 1.0))
        assert ifmm.ifmm_auto_depth(pts, lm, box) == want
    assert ifmm.ifmm_auto_depth(inputs.uniform_points(1, 10), 0) == -1


def test_blob_generator_and_batch_recipe():
    b = inputs.gaussian_blobs(11, 3000)
    assert b.shape == (3000, 2) and (b >= 0).all() and (b < 1).all()
    assert np.array_equal(b, inputs.gaussian_blobs(11, 3000))
    # clustered: the fullest of 1024 cells holds far more than the uniform mean of ~3
    cells = np.bincount((np.floor(b[:, 1] * 32) * 32 + np.floor(b[:, 0] * 32)).astype(int), minlength=1024)
    assert cells.max() > 30 and (cells == 0).sum() > 300
    sy = inputs.batch_systems(count=16)
    assert len(sy) == 16 and [s["kind"] for s in sy] == ["uniform"] * 8 + ["blobs"] * 8
    for s in sy:
        n = s["points"].shape[0]
        assert 2048 <= n <= 32768 and 1 <= s["nrhs"] <= 16
    assert len({s["points"].shape[0] for s in sy}) > 8
