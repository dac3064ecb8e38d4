"""Pins for the 3D oracle: brute force over supporting planes (exact
rationals), closed cases (cube corners plus interior points, integer points
on a sphere), Euler's formula, the inner-side invariant and permutation
invariance."""
import numpy as np
import pytest

import oracle
from tests import exact_ref as ex


def _canon(res):
    verts, faces = res
    return verts.tolist(), [tuple(f.tolist()) for f in faces]


def _tiny_sets3(seed, count):
    rng = np.random.default_rng(seed)
    for k in range(count):
        n = int(rng.integers(4, 16))
        kind = k % 4
        if kind == 0:
            p = rng.random((3, n))
        elif kind == 1:
            p = rng.integers(0, 3, (3, n))          # lattice: coplanar faces, ties
        elif kind == 2:
            base = rng.random((3, 5))
            p = base[:, rng.integers(0, 5, n)]      # duplicates
        else:
            p = rng.integers(-1, 2, (3, n)) * np.array([[1.0], [0.5], [2.0]])
        yield tuple(np.asarray(c, np.float32) for c in p)


def test_matches_brute_force():
    checked = 0
    for x, y, z in _tiny_sets3(21, 160):
        want = ex.brute_hull3d(x, y, z)
        if want is None:
            with pytest.raises(oracle.OracleError) as ei:
                oracle.hull3d(x, y, z)
            assert ei.value.code == oracle.ERR_DEGENERATE
            continue
        assert _canon(oracle.hull3d(x, y, z)) == (want[0], want[1]), (x, y, z)
        checked += 1
    assert checked > 100


def test_cube_with_interior_points():
    rng = np.random.default_rng(4)
    corners = np.array([[i, j, k] for i in (-1, 1) for j in (-1, 1) for k in (-1, 1)], np.float32)
    inner = rng.uniform(-0.99, 0.99, (3000, 3)).astype(np.float32)
    # points on the faces and edges too
    onface = rng.uniform(-1, 1, (300, 3)).astype(np.float32)
    onface[np.arange(300), rng.integers(0, 3, 300)] = rng.choice([-1.0, 1.0], 300)
    P = np.concatenate([inner, corners, onface])
    perm = rng.permutation(len(P))
    P = P[perm]
    verts, faces = oracle.hull3d(P[:, 0], P[:, 1], P[:, 2])
    assert len(verts) == 8 and len(faces) == 6
    assert all(len(f) == 4 for f in faces)
    assert np.all(np.abs(P[verts]) == 1.0)


def _euler_ok(verts, faces):
    edges = set()
    for f in faces:
        for i in range(len(f)):
            edges.add(tuple(sorted((int(f[i]), int(f[(i + 1) % len(f)])))))
    return len(verts) - len(edges) + len(faces) == 2


def test_integer_sphere_points_are_all_vertices():
    r2 = 11 ** 2 * 3  # x^2 + y^2 + z^2 = 363 has many lattice solutions
    pts = [(i, j, k) for i in range(-20, 21) for j in range(-20, 21) for k in range(-20, 21)
           if i * i + j * j + k * k == r2]
    rng = np.random.default_rng(6)
    P = np.array(pts, np.float32)[rng.permutation(len(pts))]
    inner = rng.uniform(-10, 10, (2000, 3)).astype(np.float32)
    X = np.concatenate([P, inner])
    verts, faces = oracle.hull3d(X[:, 0], X[:, 1], X[:, 2])
    assert verts.tolist() == list(range(len(P)))
    assert _euler_ok(verts, faces)


@pytest.mark.parametrize("gen", ["ball", "sphere", "gauss"])
def test_invariants(gen):
    rng = np.random.default_rng(8)
    n = 20000
    g = rng.normal(size=(3, n))
    if gen == "ball":
        g = g / np.linalg.norm(g, axis=0) * np.cbrt(rng.random(n))
    elif gen == "sphere":
        g = g / np.linalg.norm(g, axis=0)
    x, y, z = g.astype(np.float32)
    verts, faces = oracle.hull3d(x, y, z)
    assert _euler_ok(verts, faces)
    P = np.stack([x, y, z], 1)
    sample = rng.integers(0, n, 40)
    for f in faces[:: max(1, len(faces) // 60)]:
        a, b, c = P[f[0]], P[f[1]], P[f[2]]
        for i in sample:
            assert oracle.orient3d(a, b, c, P[i]) <= 0
        for v in f:  # face planar
            assert oracle.orient3d(a, b, c, P[v]) == 0
        assert f[0] == min(f)
    assert [tuple(f) for f in faces] == sorted(tuple(f) for f in faces)
    perm = rng.permutation(n)
    v2, f2 = oracle.hull3d(x[perm], y[perm], z[perm])
    assert sorted(perm[v2].tolist()) == verts.tolist()


def test_degenerate_3d():
    with pytest.raises(oracle.OracleError) as ei:
        oracle.hull3d([0, 1, 2, 3], [0, 1, 2, 3], [0, 1, 2, 3])  # collinear
    assert ei.value.code == oracle.ERR_DEGENERATE
    with pytest.raises(oracle.OracleError) as ei:
        oracle.hull3d([0, 1, 0, 1, 0.5], [0, 0, 1, 1, 0.5], [2, 2, 2, 2, 2])  # coplanar
    assert ei.value.code == oracle.ERR_DEGENERATE
    with pytest.raises(oracle.OracleError):
        oracle.hull3d([0, 1, 0], [0, 0, 1], [0, 0, 0])
    v, f = oracle.hull3d(np.zeros(0), np.zeros(0), np.zeros(0))
    assert len(v) == 0 and f == []
    # a tetrahedron
    v, f = oracle.hull3d([0, 1, 0, 0], [0, 0, 1, 0], [0, 0, 0, 1])
    assert v.tolist() == [0, 1, 2, 3]
    assert [t.tolist() for t in f] == [[0, 1, 3], [0, 2, 1], [0, 3, 2], [1, 2, 3]]


def test_batched_oracle_against_brute_force_and_closed_cases():
    # a batch mixing brute-forced tiny clouds, a cube with interior points
    # (closed form: its 8 corners and 6 square faces), an empty cloud and
    # degenerate clouds (3 points; a coplanar set); global indices
    clouds = list(_tiny_sets3(5, 24))
    rng = np.random.default_rng(9)
    corners = np.array([[i, j, k] for i in (0, 2) for j in (0, 2) for k in (0, 2)], np.float32)
    cube = np.concatenate([rng.uniform(0.1, 1.9, (40, 3)).astype(np.float32), corners])
    clouds.append(tuple(cube.T.copy()))
    clouds.append(tuple(np.zeros((3, 0), np.float32)))
    clouds.append(tuple(np.array([[0, 1, 0], [0, 0, 1], [0, 0, 0]], np.float32)))
    flat = rng.random((3, 12)).astype(np.float32)
    flat[2] = 0.5
    clouds.append(tuple(flat))
    off = np.zeros(len(clouds) + 1, np.int64)
    off[1:] = np.cumsum([len(c[0]) for c in clouds])
    x, y, z = (np.concatenate([c[i] for c in clouds]) for i in range(3))
    got = oracle.hull3d_batched(x, y, z, off)
    assert len(got) == len(clouds)
    for c, ((st, v, f), (cx, cy, cz)) in enumerate(zip(got, clouds)):
        a = int(off[c])
        if len(cx) == 0:
            assert st == oracle.OK and len(v) == 0 and f == []
            continue
        want = ex.brute_hull3d(cx, cy, cz)
        if want is None:
            assert st == oracle.ERR_DEGENERATE and len(v) == 0 and f == []
            continue
        assert st == oracle.OK
        assert (v - a).tolist() == want[0]
        assert [tuple((t - a).tolist()) for t in f] == [tuple(t) for t in want[1]]
    st, v, f = got[24]
    assert st == oracle.OK and len(v) == 8 and len(f) == 6 and all(len(t) == 4 for t in f)
    assert sorted(v.tolist()) == list(range(int(off[24]) + 40, int(off[24]) + 48))
