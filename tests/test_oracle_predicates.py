"""Pins for the oracle's exact predicates: each sign is compared with the
exact rational determinant (Python Fractions) on random and adversarial
float32 inputs, so both the FP64 filter and the exact expansion stage are
exercised."""
import numpy as np
import pytest

import oracle
from tests import exact_ref as ex


def _adversarial_2d(rng, m):
    """Triples where c lies on, or one ulp off, the line ab."""
    out = []
    for _ in range(m):
        a = rng.uniform(-1, 1, 2).astype(np.float32)
        b = rng.uniform(-1, 1, 2).astype(np.float32)
        t = rng.uniform(-2, 3)
        c = (a.astype(np.float64) + t * (b.astype(np.float64) - a)).astype(np.float32)
        k = rng.integers(-2, 3, 2)
        c = np.array([np.nextafter(c[0], np.float32(np.inf) if k[0] > 0 else np.float32(-np.inf))
                      if k[0] else c[0],
                      np.nextafter(c[1], np.float32(np.inf) if k[1] > 0 else np.float32(-np.inf))
                      if k[1] else c[1]], dtype=np.float32)
        out.append((a, b, c))
    return out


def _mixed_exponent(rng, m, d):
    out = []
    for _ in range(m):
        pts = []
        for _ in range(d + 1):
            e = rng.integers(-140, 5, d)
            v = rng.uniform(0.5, 1, d) * np.power(2.0, e) * rng.choice([-1, 1], d)
            pts.append(v.astype(np.float32))
        out.append(pts)
    return out


def test_orient2d_random_and_degenerate():
    rng = np.random.default_rng(1)
    cases = [tuple(rng.uniform(-1, 1, (3, 2)).astype(np.float32)) for _ in range(300)]
    cases += _adversarial_2d(rng, 600)
    cases += [tuple(p) for p in _mixed_exponent(rng, 300, 2)]
    # small-integer collinear and duplicate points
    for _ in range(200):
        a, b = rng.integers(-4, 5, (2, 2)).astype(np.float32)
        t = rng.integers(-3, 4)
        cases.append((a, b, (a + t * (b - a)).astype(np.float32)))
    zeros = 0
    for a, b, c in cases:
        want = ex.orient2d(a, b, c)
        zeros += want == 0
        assert oracle.orient2d(a, b, c) == want, (a, b, c)
    assert zeros > 100  # the exact stage was exercised on true zeros


def test_cmp_dist2_exact():
    rng = np.random.default_rng(2)
    n = 0
    for _ in range(800):
        a, b = rng.uniform(-1, 1, (2, 2)).astype(np.float32)
        p1 = rng.uniform(-1, 1, 2).astype(np.float32)
        if rng.random() < 0.5:
            # p2 on the parallel line through p1, possibly one ulp off
            t = rng.uniform(-1, 1)
            p2 = (p1.astype(np.float64) + t * (b.astype(np.float64) - a)).astype(np.float32)
            if rng.random() < 0.5:
                p2[1] = np.nextafter(p2[1], np.float32(2))
        else:
            p2 = rng.uniform(-1, 1, 2).astype(np.float32)
        A, B, P1, P2 = (tuple(ex.F(v) for v in q) for q in (a, b, p1, p2))
        d = (B[0] - A[0]) * (P1[1] - P2[1]) - (B[1] - A[1]) * (P1[0] - P2[0])
        want = (d > 0) - (d < 0)
        n += want == 0
        assert oracle.cmp_dist2(a, b, p1, p2) == want
    # and it really is the difference of two orientations
    for _ in range(200):
        a, b, p1, p2 = rng.uniform(-1, 1, (4, 2)).astype(np.float32)
        A, B = (tuple(ex.F(v) for v in q) for q in (a, b))
        def o(p):
            P = tuple(ex.F(v) for v in p)
            return (A[0] - P[0]) * (B[1] - P[1]) - (A[1] - P[1]) * (B[0] - P[0])
        d = o(p1) - o(p2)
        assert oracle.cmp_dist2(a, b, p1, p2) == (d > 0) - (d < 0)


def test_orient3d_random_and_coplanar():
    rng = np.random.default_rng(3)
    cases = [tuple(rng.uniform(-1, 1, (4, 3)).astype(np.float32)) for _ in range(300)]
    for _ in range(500):
        a, b, c = rng.uniform(-1, 1, (3, 3))
        s, t = rng.uniform(-2, 2, 2)
        p = (a + s * (b - a) + t * (c - a)).astype(np.float32)
        if rng.random() < 0.5:
            p[rng.integers(0, 3)] = np.nextafter(p[rng.integers(0, 3)], np.float32(9))
        cases.append((a.astype(np.float32), b.astype(np.float32), c.astype(np.float32), p))
    cases += [tuple(p) for p in _mixed_exponent(rng, 300, 3)]
    for _ in range(300):
        a, b, c = rng.integers(-3, 4, (3, 3)).astype(np.float32)
        s, t = rng.integers(-2, 3, 2)
        cases.append((a, b, c, (a + s * (b - a) + t * (c - a)).astype(np.float32)))
    zeros = 0
    for a, b, c, p in cases:
        want = ex.orient3d(a, b, c, p)
        zeros += want == 0
        assert oracle.orient3d(a, b, c, p) == want, (a, b, c, p)
    assert zeros > 100


def test_orient3d_sign_convention():
    # p above the CCW triangle (seen from +z) is positive
    a, b, c = (0, 0, 0), (1, 0, 0), (0, 1, 0)
    assert oracle.orient3d(a, b, c, (0.2, 0.2, 1)) == 1
    assert oracle.orient3d(a, b, c, (0.2, 0.2, -1)) == -1
    assert oracle.orient2d((0, 0), (1, 0), (0, 1)) == 1


def test_cmp_dist3_exact():
    rng = np.random.default_rng(4)
    for _ in range(600):
        a, b, c, p1 = rng.uniform(-1, 1, (4, 3)).astype(np.float32)
        if rng.random() < 0.5:
            s, t = rng.uniform(-1, 1, 2)
            p2 = (p1.astype(np.float64) + s * (b.astype(np.float64) - a) +
                  t * (c.astype(np.float64) - a)).astype(np.float32)
            if rng.random() < 0.5:
                p2[2] = np.nextafter(p2[2], np.float32(9))
        else:
            p2 = rng.uniform(-1, 1, 3).astype(np.float32)
        A, B, C, P1, P2 = ([ex.F(v) for v in q] for q in (a, b, c, p1, p2))
        d = ex.det3([B[i] - A[i] for i in range(3)], [C[i] - A[i] for i in range(3)],
                    [P1[i] - P2[i] for i in range(3)])
        assert oracle.cmp_dist3(a, b, c, p1, p2) == (d > 0) - (d < 0)
