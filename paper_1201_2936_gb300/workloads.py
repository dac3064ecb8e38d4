"""Seeded synthetic point clouds shared by the tests, the benchmark and the
oracle comparisons.  This module only draws numbers: it holds none of the
hull arithmetic.

Each cloud is drawn in FP64 from numpy's ``Generator(PCG64(seed))`` and cast
to float32 once; every consumer receives the same float32 buffers.  The
distributions are those of the paper's experiments (Section 5: uniform in the
circle/sphere, on it, and near it) plus the square, anisotropic-Gaussian and
batched variants used for throughput.  Arrays are structure-of-arrays: one
contiguous float32 array per coordinate.
"""
from __future__ import annotations

import numpy as np

SEED_BASE = 1201

N_SMALL_2D = 100_000
N_LARGE_2D = 16 * 1024 * 1024
N_BALL_3D = 8 * 1024 * 1024
N_SPHERE_3D = 1024 * 1024


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _soa(*cols):
    return tuple(np.ascontiguousarray(c.astype(np.float32)) for c in cols)


def uniform_square(n: int, seed: int):
    r = _rng(seed)
    return _soa(r.random(n), r.random(n))


def uniform_disk(n: int, seed: int):
    r = _rng(seed)
    rad = np.sqrt(r.random(n))
    th = 2.0 * np.pi * r.random(n)
    return _soa(rad * np.cos(th), rad * np.sin(th))


def circle_jitter(n: int, seed: int, sigma: float = 1e-4):
    r = _rng(seed)
    th = 2.0 * np.pi * r.random(n)
    rad = 1.0 + sigma * r.standard_normal(n)
    return _soa(rad * np.cos(th), rad * np.sin(th))


def on_circle(n: int, seed: int):
    return circle_jitter(n, seed, sigma=0.0)


def uniform_ball(n: int, seed: int):
    r = _rng(seed)
    g = r.standard_normal((3, n))
    g /= np.linalg.norm(g, axis=0)
    rad = np.cbrt(r.random(n))
    g *= rad
    return _soa(g[0], g[1], g[2])


def on_sphere(n: int, seed: int):
    r = _rng(seed)
    g = r.standard_normal((3, n))
    g /= np.linalg.norm(g, axis=0)
    return _soa(g[0], g[1], g[2])


def near_sphere(n: int, seed: int, sigma: float = 1e-4):
    r = _rng(seed)
    g = r.standard_normal((3, n))
    g /= np.linalg.norm(g, axis=0)
    g *= 1.0 + sigma * r.standard_normal(n)
    return _soa(g[0], g[1], g[2])


def uniform_ball_4d(n: int, seed: int):
    """Uniform in the unit 4-ball: Gaussian direction times u^(1/4)."""
    r = _rng(seed)
    g = r.standard_normal((4, n))
    g /= np.linalg.norm(g, axis=0)
    g *= r.random(n) ** 0.25
    return _soa(g[0], g[1], g[2], g[3])


def near_sphere_4d(n: int, seed: int, sigma: float = 1e-3):
    """Near the unit 3-sphere in R^4: normalised Gaussian, radius 1 + sigma N(0, 1)."""
    r = _rng(seed)
    g = r.standard_normal((4, n))
    g /= np.linalg.norm(g, axis=0)
    g *= 1.0 + sigma * r.standard_normal(n)
    return _soa(g[0], g[1], g[2], g[3])


def _random_rotation(r: np.random.Generator) -> np.ndarray:
    q, rr = np.linalg.qr(r.standard_normal((3, 3)))
    q = q * np.sign(np.diag(rr))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def batched_clouds_3d(ncloud: int, seed: int, nmin: int = 16, nmax: int = 65536):
    """Clouds with log-uniform sizes in [nmin, nmax], each an anisotropic
    Gaussian R diag(s) N(0, I) with s ~ U[0.1, 1]^3 and R a random rotation.
    Returns (x, y, z, offsets) with offsets of length ncloud + 1 (int64)."""
    r = _rng(seed)
    sizes = np.rint(np.exp(r.uniform(np.log(nmin), np.log(nmax), ncloud))).astype(np.int64)
    sizes = np.clip(sizes, nmin, nmax)
    off = np.zeros(ncloud + 1, dtype=np.int64)
    off[1:] = np.cumsum(sizes)
    pts = np.empty((3, off[-1]), dtype=np.float64)
    for c in range(ncloud):
        s = r.uniform(0.1, 1.0, 3)
        rot = _random_rotation(r)
        g = r.standard_normal((3, sizes[c]))
        pts[:, off[c]:off[c + 1]] = rot @ (s[:, None] * g)
    x, y, z = _soa(pts[0], pts[1], pts[2])
    return x, y, z, off


def batched_disk_2d(ncloud: int, npts: int, seed: int):
    r = _rng(seed)
    n = ncloud * npts
    rad = np.sqrt(r.random(n))
    th = 2.0 * np.pi * r.random(n)
    x, y = _soa(rad * np.cos(th), rad * np.sin(th))
    off = np.arange(ncloud + 1, dtype=np.int64) * npts
    return x, y, off


def batched_ball_3d(ncloud: int, npts: int, seed: int):
    x, y, z = uniform_ball(ncloud * npts, seed)
    off = np.arange(ncloud + 1, dtype=np.int64) * npts
    return x, y, z, off


# The configurations the library is measured on, by name.
CONFIGS_2D = {
    "square_100k": lambda: uniform_square(N_SMALL_2D, SEED_BASE + 0),
    "square_16M": lambda: uniform_square(N_LARGE_2D, SEED_BASE + 1),
    "disk_16M": lambda: uniform_disk(N_LARGE_2D, SEED_BASE + 11),
    "circle1e-4_16M": lambda: circle_jitter(N_LARGE_2D, SEED_BASE + 21, 1e-4),
}

CONFIGS_3D = {
    "ball_8M": lambda: uniform_ball(N_BALL_3D, SEED_BASE + 2),
    "sphere_1M": lambda: on_sphere(N_SPHERE_3D, SEED_BASE + 12),
}
