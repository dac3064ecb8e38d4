"""Pins for the 4D oracle (Section 4.3: Quickhull in higher dimensions).

The exact orientation and distance comparison against rational arithmetic;
the hull against a brute force over supporting hyperplanes in exact
rationals (random, lattice and duplicated tiny inputs); closed cases: the
tesseract's 16 corners with interior and boundary points (16 vertices, 8
cubic facets), the cross-polytope (8 vertices, 16 tetrahedra), integer points
on a 3-sphere (all vertices); Euler's relation f0 - f1 + f2 - f3 = 0 for
simplicial hulls; every point on the inner side of every facet; permutation
invariance; degenerate inputs."""
from itertools import combinations

import numpy as np
import pytest

import oracle
from paper_1201_2936_gb300 import workloads as w
from tests import exact_ref as ex


def _canon(res):
    verts, facets = res
    return verts.tolist(), [tuple(f.tolist()) for f in facets]


def test_orient4_matches_rationals():
    rng = np.random.default_rng(41)
    for k in range(400):
        if k % 3 == 0:
            P = rng.standard_normal((5, 4)).astype(np.float32)
        elif k % 3 == 1:
            # p on the hyperplane of a, b, c, d (affine combination), nudged by
            # an ulp or not at all
            Q = rng.integers(-8, 8, (4, 4)).astype(np.float32)
            wts = rng.integers(-3, 4, 3)
            p = Q[0] + wts[0] * (Q[1] - Q[0]) + wts[1] * (Q[2] - Q[0]) + wts[2] * (Q[3] - Q[0])
            p = p.astype(np.float32)
            if k % 2:
                i = rng.integers(0, 4)
                p[i] = np.nextafter(p[i], np.float32(np.inf))
            P = np.vstack([Q, p[None, :]])
        else:
            # mixed exponents
            P = (rng.standard_normal((5, 4)) *
                 np.exp2(rng.integers(-60, 60, (5, 4)))).astype(np.float32)
        a, b, c, d, p = (P[i] for i in range(5))
        assert oracle.orient4(a, b, c, d, p) == ex.orient4(a, b, c, d, p), P


def test_cmp_dist4_matches_rationals():
    rng = np.random.default_rng(42)
    for k in range(300):
        P = rng.standard_normal((6, 4)).astype(np.float32)
        if k % 2:
            # equal distance: p2 = p1 plus a vector inside the hyperplane
            P[5] = (P[4] + (P[1] - P[0]) * 2 - (P[2] - P[0])).astype(np.float32)
        a, b, c, d, p1, p2 = (P[i] for i in range(6))
        A, B, C, D, P1, P2 = ([ex.F(t) for t in q] for q in (a, b, c, d, p1, p2))
        rows = [[B[i] - A[i] for i in range(4)], [C[i] - A[i] for i in range(4)],
                [D[i] - A[i] for i in range(4)], [P1[i] - P2[i] for i in range(4)]]
        v = ex.det4(rows)
        assert oracle.cmp_dist4(a, b, c, d, p1, p2) == (v > 0) - (v < 0)


def _tiny_sets4(seed, count):
    rng = np.random.default_rng(seed)
    for k in range(count):
        n = int(rng.integers(5, 13))
        kind = k % 4
        if kind == 0:
            p = rng.random((4, n))
        elif kind == 1:
            p = rng.integers(0, 3, (4, n))          # lattice: cohyperplanar facets, ties
        elif kind == 2:
            base = rng.random((4, 6))
            p = base[:, rng.integers(0, 6, n)]      # duplicates
        else:
            p = rng.integers(-1, 2, (4, n)) * np.array([[1.0], [0.5], [2.0], [0.25]])
        yield tuple(np.asarray(c, np.float32) for c in p)


def test_matches_brute_force():
    checked = 0
    for x, y, z, ww in _tiny_sets4(51, 120):
        want = ex.brute_hull4d(x, y, z, ww)
        if want is None:
            with pytest.raises(oracle.OracleError) as ei:
                oracle.hull4d(x, y, z, ww)
            assert ei.value.code == oracle.ERR_DEGENERATE
            continue
        assert _canon(oracle.hull4d(x, y, z, ww)) == (want[0], want[1]), (x, y, z, ww)
        checked += 1
    assert checked > 60


def test_tesseract_with_interior_and_boundary_points():
    rng = np.random.default_rng(7)
    corners = np.array([[i, j, k, l] for i in (-1, 1) for j in (-1, 1) for k in (-1, 1)
                        for l in (-1, 1)], np.float32)
    inner = rng.uniform(-0.99, 0.99, (4000, 4)).astype(np.float32)
    # points on the facets, 2-faces and edges: not vertices
    bnd = rng.uniform(-1, 1, (400, 4)).astype(np.float32)
    for r in range(400):
        fix = rng.choice(4, size=int(rng.integers(1, 4)), replace=False)
        bnd[r, fix] = rng.choice([-1.0, 1.0], len(fix))
    P = np.concatenate([bnd, inner, corners])
    P = P[rng.permutation(len(P))]
    verts, facets = oracle.hull4d(P[:, 0], P[:, 1], P[:, 2], P[:, 3])
    assert len(verts) == 16 and np.all(np.abs(P[verts]) == 1.0)
    assert len(facets) == 8 and all(len(f) == 8 for f in facets)
    for f in facets:  # each facet is a cube: one coordinate fixed at +-1
        c = P[f]
        assert any(np.all(c[:, k] == c[0, k]) for k in range(4))


def _euler_simplicial(verts, facets):
    e, t = set(), set()
    for f in facets:
        assert len(f) == 4
        for a, b in combinations(f, 2):
            e.add((a, b))
        for tri in combinations(f, 3):
            t.add(tri)
    return len(verts) - len(e) + len(t) - len(facets) == 0


def test_cross_polytope():
    rng = np.random.default_rng(8)
    tips = np.vstack([np.eye(4), -np.eye(4)]).astype(np.float32)
    inner = rng.uniform(-0.2, 0.2, (500, 4)).astype(np.float32)
    P = np.concatenate([inner, tips])
    verts, facets = oracle.hull4d(P[:, 0], P[:, 1], P[:, 2], P[:, 3])
    assert verts.tolist() == list(range(500, 508))
    assert len(facets) == 16
    assert _euler_simplicial(verts.tolist(), [tuple(f) for f in facets])


def test_integer_points_on_a_3_sphere_are_all_vertices():
    r2 = 27
    pts = [(a, b, c, d) for a in range(-5, 6) for b in range(-5, 6) for c in range(-5, 6)
           for d in range(-5, 6) if a * a + b * b + c * c + d * d == r2]
    P = np.array(pts, np.float32)
    # interior points well inside: the ball of radius 2.5 (the lattice
    # points' hull holds far more than that around the origin)
    inner = 2.5 * np.stack(w.uniform_ball_4d(2000, 9), axis=1)
    Q = np.concatenate([P, inner.astype(np.float32)])
    verts, facets = oracle.hull4d(Q[:, 0], Q[:, 1], Q[:, 2], Q[:, 3])
    assert verts.tolist() == list(range(len(P)))


def _inner_side_ok(P, facets):
    for f in facets:
        a, b, c, d = (P[i] for i in f[:4])
        s = {oracle.orient4(a, b, c, d, p) for p in P}
        if not (s <= {0, 1} or s <= {0, -1}):
            return False
    return True


@pytest.mark.parametrize("gen", ["ball", "near"])
def test_general_position_invariants(gen):
    n = 3000
    x, y, z, ww = (w.uniform_ball_4d(n, 61) if gen == "ball" else w.near_sphere_4d(n, 62, 1e-3))
    verts, facets = oracle.hull4d(x, y, z, ww)
    assert all(len(f) == 4 for f in facets)
    assert _euler_simplicial(verts.tolist(), [tuple(f) for f in facets])
    P = np.stack([x, y, z, ww], axis=1)
    sample = facets[:: max(1, len(facets) // 150)]
    assert _inner_side_ok(P, sample)
    # the vertices are exactly the points on some facet
    assert sorted({int(i) for f in facets for i in f}) == verts.tolist()


def test_permutation_invariance():
    x, y, z, ww = w.uniform_ball_4d(1500, 63)
    v0, f0 = oracle.hull4d(x, y, z, ww)
    perm = np.random.default_rng(64).permutation(len(x))
    v1, f1 = oracle.hull4d(x[perm], y[perm], z[perm], ww[perm])
    back = sorted(perm[v1].tolist())
    assert back == v0.tolist()
    assert sorted(tuple(sorted(perm[f].tolist())) for f in f1) == [tuple(f) for f in
                                                                   (t.tolist() for t in f0)]


def test_degenerate_inputs():
    rng = np.random.default_rng(10)
    p = rng.random((3, 50)).astype(np.float32)
    with pytest.raises(oracle.OracleError) as ei:   # all in the hyperplane w = 0.5
        oracle.hull4d(p[0], p[1], p[2], np.full(50, 0.5, np.float32))
    assert ei.value.code == oracle.ERR_DEGENERATE
    with pytest.raises(oracle.OracleError) as ei:
        oracle.hull4d(*rng.random((4, 4)).astype(np.float32))
    assert ei.value.code == oracle.ERR_DEGENERATE
    v, f = oracle.hull4d(*(np.zeros(0, np.float32) for _ in range(4)))
    assert len(v) == 0 and len(f) == 0
    bad = rng.random((4, 10)).astype(np.float32)
    bad[2, 3] = np.nan
    with pytest.raises(oracle.OracleError) as ei:
        oracle.hull4d(*bad)
    assert ei.value.code == oracle.ERR_NONFINITE
