"""The seeded generators are deterministic and produce the stated shapes."""
import numpy as np

from paper_1201_2936_gb300 import workloads as w


def test_deterministic_and_float32():
    a = w.uniform_disk(1000, 7)
    b = w.uniform_disk(1000, 7)
    assert all(np.array_equal(p, q) for p, q in zip(a, b))
    assert all(c.dtype == np.float32 and c.flags.c_contiguous for c in a)
    assert np.all(a[0] ** 2 + a[1] ** 2 <= 1.0 + 1e-6)


def test_distributions():
    x, y = w.circle_jitter(20000, 3, 1e-4)
    r = np.hypot(x.astype(np.float64), y.astype(np.float64))
    assert abs(np.std(r) - 1e-4) < 1e-5
    x, y, z = w.on_sphere(5000, 4)
    r = np.sqrt(x.astype(np.float64) ** 2 + y ** 2 + z ** 2)
    assert np.max(np.abs(r - 1)) < 1e-6
    x, y, z, off = w.batched_clouds_3d(64, 5)
    sizes = np.diff(off)
    assert len(sizes) == 64 and sizes.min() >= 16 and sizes.max() <= 65536
    assert len(x) == off[-1]


def _frac_within(r, t):
    return float(np.mean(r <= t))


def test_radial_laws_of_the_uniform_regions():
    # uniform in the unit d-ball: P(|p| <= t) = t^d; the tolerance is five
    # binomial standard deviations at n = 200k
    n = 200_000
    tol = 5 * np.sqrt(0.25 / n)
    x, y = w.uniform_square(n, 11)
    assert x.min() >= 0 and x.max() < 1 and y.min() >= 0 and y.max() < 1
    assert abs(_frac_within(x, 0.5) - 0.5) < tol and abs(_frac_within(y, 0.25) - 0.25) < tol
    cases = [(2, w.uniform_disk(n, 12)), (3, w.uniform_ball(n, 13)), (4, w.uniform_ball_4d(n, 14))]
    for d, cols in cases:
        r = np.sqrt(sum(c.astype(np.float64) ** 2 for c in cols))
        assert r.max() <= 1 + 1e-6, d
        for t in (0.5, 0.8, 0.95):
            assert abs(_frac_within(r, t) - t ** d) < tol, (d, t)
        # directions: every coordinate's mean is near zero and its sign balanced
        for c in cols:
            assert abs(float(np.mean(c > 0)) - 0.5) < tol, d


def test_radial_jitter_widths():
    n = 100_000
    for sigma, cols in ((1e-4, w.near_sphere(n, 15, 1e-4)), (1e-3, w.near_sphere_4d(n, 16)),
                        (1e-2, w.near_sphere_4d(n, 17, 1e-2))):
        r = np.sqrt(sum(c.astype(np.float64) ** 2 for c in cols))
        # float32 rounding of the coordinates adds ~6e-8 of radial noise
        assert abs(np.std(r) - sigma) < 0.02 * sigma + 1e-7, sigma
        assert abs(np.mean(r) - 1.0) < 5 * sigma / np.sqrt(n) + 1e-7, sigma
    x, y = w.on_circle(10_000, 18)
    assert np.max(np.abs(np.hypot(x.astype(np.float64), y) - 1)) < 1e-6


def test_batched_clouds_sizes_and_shapes():
    # log-uniform sizes in [nmin, nmax]; each cloud an anisotropic Gaussian
    # whose covariance has eigenvalues s_i^2 with s_i in [0.1, 1]
    x, y, z, off = w.batched_clouds_3d(512, 19, nmin=16, nmax=4096)
    sizes = np.diff(off)
    assert sizes.min() >= 16 and sizes.max() <= 4096 and len(x) == off[-1]
    logs = np.log(sizes)
    lo, hi = np.log(16), np.log(4096)
    assert abs(logs.mean() - (lo + hi) / 2) < 5 * (hi - lo) / np.sqrt(12 * 512)
    assert abs(float(np.mean(logs <= (lo + hi) / 2)) - 0.5) < 5 * np.sqrt(0.25 / 512)
    big = np.argsort(sizes)[-8:]
    for c in big:
        P = np.stack([x[off[c]:off[c + 1]], y[off[c]:off[c + 1]], z[off[c]:off[c + 1]]])
        ev = np.linalg.eigvalsh(np.cov(P.astype(np.float64)))
        assert ev.min() > 0.01 * 0.8 and ev.max() < 1.0 * 1.25, (c, ev)
    # fixed-size batches: equal shares and the stated per-cloud laws
    x, y, off = w.batched_disk_2d(16, 1000, 20)
    assert list(np.diff(off)) == [1000] * 16 and len(x) == 16_000
    x, y, z, off = w.batched_ball_3d(8, 500, 21)
    assert list(np.diff(off)) == [500] * 8
    assert np.sqrt(x.astype(np.float64) ** 2 + y ** 2 + z ** 2).max() <= 1 + 1e-6
