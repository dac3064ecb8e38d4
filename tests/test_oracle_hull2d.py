"""Pins for the 2D oracle: brute force (O(n^3) edge test, exact rationals),
Andrew's monotone chain with exact orientation, closed cases (integer points
on a circle are all vertices), degenerate inputs and invariants."""
import math

import numpy as np
import pytest

import oracle
from tests import exact_ref as ex


def _tiny_sets(seed, count):
    rng = np.random.default_rng(seed)
    for k in range(count):
        n = int(rng.integers(1, 28))
        kind = k % 5
        if kind == 0:
            x, y = rng.random((2, n))
        elif kind == 1:      # small integer grid: collinear runs, duplicates, ties
            x, y = rng.integers(0, 4, (2, n))
        elif kind == 2:      # all collinear
            t = rng.integers(-5, 6, n)
            x, y = 2 * t + 1, -t
        elif kind == 3:      # duplicates of a few locations
            base = rng.random((2, 4))
            pick = rng.integers(0, 4, n)
            x, y = base[0, pick], base[1, pick]
        else:                # a rectangle with points on its sides
            x = rng.integers(0, 3, n) * 0.5
            y = rng.choice([0.0, 1.0], n)
        yield np.asarray(x, np.float32), np.asarray(y, np.float32)


def test_matches_brute_force_and_monotone_chain():
    for x, y in _tiny_sets(11, 400):
        got = oracle.hull2d(x, y).tolist()
        assert got == ex.brute_hull2d(x, y), (x, y)
        assert got == ex.monotone_chain2d(x, y), (x, y)


@pytest.mark.parametrize("n,seed", [(200, 1), (2000, 2), (5000, 3)])
def test_matches_monotone_chain_larger(n, seed):
    rng = np.random.default_rng(seed)
    x, y = rng.random((2, n)).astype(np.float32)
    assert oracle.hull2d(x, y).tolist() == ex.monotone_chain2d(x, y)
    x, y = rng.normal(size=(2, n)).astype(np.float32)
    assert oracle.hull2d(x, y).tolist() == ex.monotone_chain2d(x, y)


def test_integer_circle_points_are_all_vertices():
    # all lattice points on x^2 + y^2 = r^2 with r = 5^3 = 125 are extreme
    r = 125
    pts = [(i, j) for i in range(-r, r + 1) for j in (int(math.isqrt(r * r - i * i)),)
           if j * j == r * r - i * i]
    pts = sorted({(i, s * j) for i, j in pts for s in (1, -1)})
    rng = np.random.default_rng(5)
    perm = rng.permutation(len(pts))
    x = np.array([pts[p][0] for p in perm], np.float32)
    y = np.array([pts[p][1] for p in perm], np.float32)
    # add interior points
    xi, yi = rng.uniform(-80, 80, (2, 500)).astype(np.float32)
    X, Y = np.concatenate([x, xi]), np.concatenate([y, yi])
    got = oracle.hull2d(X, Y)
    assert sorted(got.tolist()) == list(range(len(pts)))
    # counter-clockwise: positive signed area, starting at the lexicographic min
    hx, hy = X[got].astype(np.float64), Y[got].astype(np.float64)
    area = 0.5 * np.sum(hx * np.roll(hy, -1) - np.roll(hx, -1) * hy)
    assert area > 0
    assert (hx[0], hy[0]) == min(zip(hx, hy))


def test_degenerate_cases():
    e = np.zeros(0, np.float32)
    assert oracle.hull2d(e, e).tolist() == []
    assert oracle.hull2d([3.0], [4.0]).tolist() == [0]
    assert oracle.hull2d([1, 1, 1], [2, 2, 2]).tolist() == [0]
    # collinear: the two extreme points, lexicographic min first
    assert oracle.hull2d([2, 0, 1, 3], [2, 0, 1, 3]).tolist() == [1, 3]
    # duplicates of a vertex report the lowest index
    assert oracle.hull2d([0, 1, 0, 1, 1, 0], [0, 0, 1, 1, 0, 0]).tolist() == [0, 1, 3, 2]
    # -0.0 and +0.0 are the same location
    assert oracle.hull2d([0.0, -0.0, 1.0, 0.0], [0.0, 0.0, 0.0, 1.0]).tolist() == [0, 2, 3]
    with pytest.raises(oracle.OracleError) as ei:
        oracle.hull2d([0.0, np.nan], [0.0, 1.0])
    assert ei.value.code == oracle.ERR_NONFINITE
    with pytest.raises(oracle.OracleError):
        oracle.hull2d([0.0, 1.0], [np.inf, 1.0])


def test_invariants_and_permutation():
    rng = np.random.default_rng(9)
    x, y = rng.normal(size=(2, 20000)).astype(np.float32)
    h = oracle.hull2d(x, y)
    P = np.stack([x, y], 1)
    # every input point is on the inner side of (or on) every hull edge
    m = len(h)
    for k in range(m):
        a, b = P[h[k]], P[h[(k + 1) % m]]
        s = np.array([oracle.orient2d(a, b, P[i]) for i in rng.integers(0, len(x), 300)])
        assert np.all(s >= 0)
        assert oracle.orient2d(P[h[k - 1]], a, b) > 0   # strict convexity
    perm = rng.permutation(len(x))
    h2 = oracle.hull2d(x[perm], y[perm])
    assert sorted(perm[h2].tolist()) == sorted(h.tolist())
