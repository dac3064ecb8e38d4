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
