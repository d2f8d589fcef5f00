"""The seeded input generators (paper_1407_1572_gb300/inputs.py) against their published
definitions: SplitMix64's first outputs for seed 0 are the values listed with the generator's
reference implementation (Steele, Lea and Flood; Vigna's splitmix64.c); the uniforms are the top 53
bits scaled into [0, 1); Box-Muller normals have zero mean and unit variance."""
import numpy as np

from paper_1407_1572_gb300 import inputs


def test_splitmix64_matches_the_published_sequence():
    assert [int(v) for v in inputs.splitmix64(0, 3)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
                                                          0x06C45D188009454F]


def test_splitmix64_streams_are_consecutive():
    # the stream of seed s + k * golden continues the stream of seed s after k outputs
    a = inputs.splitmix64(1407, 10)
    b = inputs.splitmix64((1407 + 4 * 0x9E3779B97F4A7C15) & ((1 << 64) - 1), 6)
    assert np.array_equal(a[4:], b)


def test_uniforms_are_the_top_53_bits():
    z = inputs.splitmix64(7, 1000)
    u = inputs.uniform(7, 1000)
    assert np.array_equal(u, (z >> np.uint64(11)).astype(np.float64) / 2.0 ** 53)
    assert u.min() >= 0.0 and u.max() < 1.0


def test_normals_have_unit_variance_and_points_fill_the_box():
    z = inputs.normal(11, 200_000)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01
    p = inputs.uniform_points(3, 50_000, lo=-1.0, side=2.0)
    assert p.min() >= -1.0 and p.max() < 1.0
    assert np.allclose(np.histogram(p[:, 0], bins=4, range=(-1, 1))[0] / 50_000, 0.25, atol=0.01)
