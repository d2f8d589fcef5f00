"""Seeded synthetic inputs shared by the tests, the bench, the CUDA path and the oracle.

This module holds no arithmetic of the method: only the random streams that produce points and
right-hand sides, so that both sides of a parity test see identical inputs.

Generator: SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014) -> 53-bit uniforms in [0, 1); normals by the Box-Muller transform.
Workloads follow the paper's 2D benchmarks (Section 5: points drawn at random in a square, a
balanced tree): points i.i.d. uniform in the unit square, right-hand sides i.i.d. N(0, 1).
"""
from __future__ import annotations

import numpy as np

_MASK = (1 << 64) - 1
_GOLDEN = 0x9E3779B97F4A7C15


def splitmix64(seed: int, count: int) -> np.ndarray:
    """`count` consecutive SplitMix64 outputs of the stream started at `seed` (uint64)."""
    idx = np.arange(1, count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & _MASK) + idx * np.uint64(_GOLDEN)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, count: int) -> np.ndarray:
    """53-bit uniforms in [0, 1)."""
    return (splitmix64(seed, count) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def normal(seed: int, count: int) -> np.ndarray:
    """Standard normals by Box-Muller on pairs of uniforms."""
    m = (count + 1) // 2
    u = uniform(seed, 2 * m)
    u1 = 1.0 - u[0::2]  # (0, 1]
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    z = np.empty(2 * m)
    z[0::2] = rad * np.cos(2.0 * np.pi * u2)
    z[1::2] = rad * np.sin(2.0 * np.pi * u2)
    return z[:count]


def uniform_points(seed: int, n: int, lo: float = 0.0, side: float = 1.0) -> np.ndarray:
    """n points i.i.d. uniform in [lo, lo+side)^2, shape (n, 2) float64."""
    u = uniform(seed, 2 * n).reshape(n, 2)
    return lo + side * u


def gaussian_blobs(seed: int, n: int, k: int = 8, sigma: float = 0.05, lo: float = 0.15, hi: float = 0.85) -> np.ndarray:
    """n points from an equal-weight mixture of k isotropic Gaussians of standard deviation sigma whose
    centres are uniform in [lo, hi]^2; a draw outside [0, 1)^2 is drawn again. Shape (n, 2)."""
    centres = lo + (hi - lo) * uniform(seed, 2 * k).reshape(k, 2)
    out = np.empty((n, 2))
    filled, attempt = 0, 0
    while filled < n:
        m = 2 * (n - filled) + 16
        s = seed + 7919 * (attempt + 1)
        comp = np.minimum((uniform(s, m) * k).astype(np.int64), k - 1)
        cand = centres[comp] + sigma * normal(s + 1, 2 * m).reshape(m, 2)
        ok = (cand >= 0.0).all(axis=1) & (cand < 1.0).all(axis=1)
        take = cand[ok][: n - filled]
        out[filled: filled + len(take)] = take
        filled += len(take)
        attempt += 1
    return out


def batch_systems(seed: int = 1409, count: int = 256, nmin: int = 2048, nmax: int = 32768, rhs_min: int = 1,
                  rhs_max: int = 16) -> list:
    """The batched workload: `count` independent systems with N log-uniform in [nmin, nmax]; the first
    half of the systems are uniform point clouds, the second half Gaussian blobs (8 centres, sigma
    0.05); nrhs uniform in [rhs_min, rhs_max]. System i draws its points and right-hand sides from
    seed * 1000 + i. Returns dicts with keys points, nrhs, kind, seed."""
    u = uniform(seed, 2 * count)
    out = []
    for i in range(count):
        n = int(round(float(np.exp(np.log(nmin) + (np.log(nmax) - np.log(nmin)) * u[2 * i]))))
        nrhs = rhs_min + min(int(u[2 * i + 1] * (rhs_max - rhs_min + 1)), rhs_max - rhs_min)
        si = seed * 1000 + i
        kind = "uniform" if i < count // 2 else "blobs"
        pts = uniform_points(si, n) if kind == "uniform" else gaussian_blobs(si, n)
        out.append(dict(points=pts, nrhs=nrhs, kind=kind, seed=si))
    return out


def rhs(seed: int, n: int, nrhs: int) -> np.ndarray:
    """n x nrhs right-hand sides i.i.d. N(0, 1), column-major (Fortran) float64."""
    return np.asfortranarray(normal(seed, n * nrhs).reshape(nrhs, n).T)


# Workloads named by what they are; seeds are 1407 + workload index.
WORKLOADS = {
    "n4096_d3_p4": dict(N=4096, depth=3, cheb_p=4, eps=1e-10, nrhs=1, seed=1407),
    "n65536_d5_p4": dict(N=65536, depth=5, cheb_p=4, eps=1e-6, nrhs=8, seed=1408),
    "n65536_d5_p6": dict(N=65536, depth=5, cheb_p=6, eps=1e-6, nrhs=8, seed=1408),
    "n1048576_d7_p4": dict(N=1048576, depth=7, cheb_p=4, eps=1e-6, nrhs=32, seed=1411),
}
