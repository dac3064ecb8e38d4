"""GPU parity for the 3D hull: vertex list and canonical face list of the
CUDA path (through the C ABI) equal the oracle's, on seeded inputs of the
paper's distributions (in, on, near the sphere), Gaussian clouds, lattices
with coplanar faces and collinear edges, and degenerate inputs."""
import numpy as np
import pytest
import torch

import oracle
from paper_1201_2936_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qh():
    from paper_1201_2936_gb300 import build
    build.build()
    oracle.build()
    import paper_1201_2936_gb300 as q
    return q


def _gpu(qh, x, y, z, **kw):
    X, Y, Z = (torch.from_numpy(np.ascontiguousarray(c, dtype=np.float32)).cuda() for c in (x, y, z))
    (v, off, idx), res = qh.hull3d(X, Y, Z, return_result=True, **kw)
    v, off, idx = v.cpu().numpy(), off.cpu().numpy(), idx.cpu().numpy()
    faces = [idx[off[i]:off[i + 1]].tolist() for i in range(len(off) - 1)]
    return v.tolist(), faces, res


def _oracle(x, y, z):
    v, f = oracle.hull3d(x, y, z)
    return v.tolist(), [t.tolist() for t in f]


@pytest.mark.parametrize("gen,n", [("ball", 1000), ("ball", 100_003), ("sphere", 20_000),
                                   ("near", 50_000), ("gauss", 200_001), ("ball", 5)])
def test_distributions_match_oracle(qh, gen, n):
    seed = 300 + n
    if gen == "ball":
        x, y, z = w.uniform_ball(n, seed)
    elif gen == "sphere":
        x, y, z = w.on_sphere(n, seed)
    elif gen == "near":
        x, y, z = w.near_sphere(n, seed, 1e-3)
    else:
        r = np.random.default_rng(seed)
        x, y, z = (r.normal(size=(3, n)) * np.array([[1.0], [0.3], [2.0]])).astype(np.float32)
    want = _oracle(x, y, z)
    for pred in ("f32", "f64"):
        v, f, res = _gpu(qh, x, y, z, pred=pred)
        assert v == want[0], (gen, n, pred)
        assert f == want[1], (gen, n, pred)


def test_cube_lattice_and_coplanar(qh):
    rng = np.random.default_rng(7)
    corners = np.array([[i, j, k] for i in (-1, 1) for j in (-1, 1) for k in (-1, 1)], np.float32)
    inner = rng.uniform(-0.99, 0.99, (5000, 3)).astype(np.float32)
    onface = rng.uniform(-1, 1, (500, 3)).astype(np.float32)
    onface[np.arange(500), rng.integers(0, 3, 500)] = rng.choice([-1.0, 1.0], 500)
    P = np.concatenate([inner, corners, onface])[rng.permutation(5508)]
    want = _oracle(P[:, 0], P[:, 1], P[:, 2])
    v, f, _ = _gpu(qh, P[:, 0], P[:, 1], P[:, 2])
    assert (v, f) == (want[0], want[1])
    assert len(f) == 6
    for k in range(6):  # small lattices: many coplanar facets and ties
        P = rng.integers(-3, 4, (400 + 50 * k, 3)).astype(np.float32)
        want = _oracle(P[:, 0], P[:, 1], P[:, 2])
        v, f, _ = _gpu(qh, P[:, 0], P[:, 1], P[:, 2])
        assert (v, f) == (want[0], want[1]), k


def test_degenerate_inputs(qh):
    for pts in ([[0, 0, 0], [1, 1, 1], [2, 2, 2], [3, 3, 3]],
                [[0, 0, 2], [1, 0, 2], [0, 1, 2], [1, 1, 2], [0.5, 0.5, 2]],
                [[1, 2, 3]] * 10):
        P = np.array(pts, np.float32)
        with pytest.raises(qh.QHError) as ei:
            _gpu(qh, P[:, 0], P[:, 1], P[:, 2])
        assert ei.value.status == 3
    P = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float32)
    v, f, _ = _gpu(qh, P[:, 0], P[:, 1], P[:, 2])
    assert (v, f) == _oracle(P[:, 0], P[:, 1], P[:, 2])


def test_interleaved_layout(qh):
    x, y, z = w.uniform_ball(30_000, 11)
    want = _oracle(x, y, z)
    P = torch.from_numpy(np.stack([x, y, z], 1)).cuda()
    v, off, idx = qh.hull3d(P)
    faces = [idx[off[i]:off[i + 1]].tolist() for i in range(len(off) - 1)]
    assert v.tolist() == want[0] and faces == want[1]


@pytest.mark.parametrize("gen", ["ball8M", "sphere1M"])
def test_full_size_matches_oracle(qh, gen):
    # the 3D benchmark workloads at full size, in the launch configuration the
    # benchmark times (persistent kernel, both predicate modes)
    if gen == "ball8M":
        x, y, z = w.uniform_ball(w.N_BALL_3D, w.SEED_BASE + 2)
    else:
        x, y, z = w.on_sphere(w.N_SPHERE_3D, w.SEED_BASE + 12)
    ov, of = oracle.hull3d(x, y, z)
    oo = np.zeros(len(of) + 1, np.int64)
    oo[1:] = np.cumsum([len(f) for f in of])
    oi = np.concatenate(of)
    X, Y, Z = (torch.from_numpy(c).cuda() for c in (x, y, z))
    for pred in ("f32", "f64"):
        v, off, idx = qh.hull3d(X, Y, Z, pred=pred)
        assert np.array_equal(v.cpu().numpy(), ov), pred
        assert np.array_equal(off.cpu().numpy(), oo), pred
        assert np.array_equal(idx.cpu().numpy(), oi), pred


def _paraboloid_dup_huge():
    r = np.random.default_rng(61)
    # integer paraboloid z = x^2 + y^2: the four points of every grid cell
    # are coplanar, and the farthest points of many facets tie exactly
    i, j = np.meshgrid(np.arange(-30, 31), np.arange(-30, 31))
    i, j = i.ravel(), j.ravel()
    ix, iy = r.integers(-29, 30, (2, 20_000))
    iz = ix * ix + iy * iy + 1 + r.integers(0, 500, 20_000)
    P = np.concatenate([np.stack([i, j, i * i + j * j], 1),
                        np.stack([ix, iy, np.minimum(iz, 1799)], 1)]).astype(np.float32)
    P = P[r.permutation(len(P))]
    para = (P[:, 0].copy(), P[:, 1].copy(), P[:, 2].copy())
    # hull vertices of a ball repeated at lower and higher indices
    bx, by, bz = w.uniform_ball(40_000, 62)
    hv = oracle.hull3d(bx, by, bz)[0][:16]
    dup = tuple(np.concatenate([c[hv], c, c[hv]]).astype(np.float32) for c in (bx, by, bz))
    # coordinates near 1e13: the FP32 orientation overflows, the exact path decides
    hx, hy, hz = w.uniform_ball(20_000, 63)
    huge = tuple((c * np.float32(1e13)).astype(np.float32) for c in (hx, hy, hz))
    return [para, dup, huge]


@pytest.mark.parametrize("pred", ["f32", "f64"])
def test_exact_ties_duplicates_and_filter_overflow(qh, pred):
    for k, (x, y, z) in enumerate(_paraboloid_dup_huge()):
        want = _oracle(x, y, z)
        v, f, _ = _gpu(qh, x, y, z, pred=pred)
        assert (v, f) == (want[0], want[1]), (k, pred)


def test_non_finite_input(qh):
    x, y, z = w.uniform_ball(1000, 64)
    for bad in (np.nan, np.inf):
        zz = z.copy()
        zz[123] = bad
        with pytest.raises(qh.QHError) as ei:
            _gpu(qh, x, y, zz)
        assert ei.value.status == 2


def test_near_sphere_full_size(qh):
    # the benchmark's near-sphere workload at full size (8M points, radius
    # 1 + 1e-4 N(0, 1)): vertex list and faces equal the oracle's
    x, y, z = w.near_sphere(w.N_BALL_3D, w.SEED_BASE + 22, 1e-4)
    gv, gf, res = _gpu(qh, x, y, z)
    ov, of = _oracle(x, y, z)
    assert res["status"] == 0
    assert gv == ov
    assert gf == of


def test_first_polytope_extreme_copies_and_signed_zeros(qh):
    # the single-cloud first polytope starts from each direction's extreme
    # point (axes and diagonals): put copies of those points at lower and
    # higher indices, with -0.0 in place of 0.0 in some copies, so that each
    # direction's maximum ties across copies (the lowest index must win, as
    # in the oracle)
    rng = np.random.default_rng(64)
    inner = (0.8 * np.stack(w.uniform_ball(30_000, 65), axis=1)).astype(np.float32)
    ext = np.array([[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1],
                    [.6, .6, .5], [-.6, .6, .5], [.6, -.6, .5], [-.6, -.6, .5],
                    [.6, .6, -.5], [-.6, .6, -.5], [.6, -.6, -.5], [-.6, -.6, -.5]], np.float32)
    negz = ext.copy()
    negz[negz == 0] = np.float32(-0.0)
    P = np.concatenate([negz[rng.permutation(14)], inner, ext, negz])
    for perm in (np.arange(len(P)), rng.permutation(len(P))):
        Q = P[perm]
        want = _oracle(Q[:, 0], Q[:, 1], Q[:, 2])
        for pred in ("f32", "f64"):
            v, f, _ = _gpu(qh, Q[:, 0], Q[:, 1], Q[:, 2], pred=pred)
            assert (v, f) == (want[0], want[1]), pred


@pytest.mark.parametrize("scale", [1e-20, 1e-30])
def test_filter_underflow_scales(qh, scale):
    # products of coordinate differences below FP32's normal range: the
    # filters must not decide on underflowed values
    x, y, z = w.uniform_ball(60_000, 66)
    s = np.float32(scale)
    X, Y, Z = ((c * s).astype(np.float32) for c in (x, y, z))
    want = _oracle(X, Y, Z)
    for pred in ("f32", "f64"):
        v, f, _ = _gpu(qh, X, Y, Z, pred=pred)
        assert (v, f) == (want[0], want[1]), pred


def test_every_point_twice_and_signed_zeros(qh):
    rng = np.random.default_rng(68)
    pts = np.stack(w.uniform_ball(50_000, 69), axis=1).astype(np.float32)
    pts[rng.integers(0, 50_000, 2_000), rng.integers(0, 3, 2_000)] = np.float32(0.0)
    twin = pts.copy()
    twin[twin == 0] = np.float32(-0.0)
    P = np.concatenate([pts, twin, pts[rng.permutation(50_000)]])
    want = _oracle(P[:, 0], P[:, 1], P[:, 2])
    for pred in ("f32", "f64"):
        v, f, _ = _gpu(qh, P[:, 0], P[:, 1], P[:, 2], pred=pred)
        assert (v, f) == (want[0], want[1]), pred


@pytest.mark.parametrize("offset", [0.0, 1000.0])
def test_first_polytope_facet_boundary(qh, offset):
    # The single-cloud first assignment sends each point to the first facet
    # of the first polytope (the extreme points of the axes and diagonals)
    # that it is strictly above.  One hull vertex just outside each facet
    # (1e-5 of its distance from the facet vertices' mean beyond the facet),
    # interior points filling the ball of the nearest facet's distance up to
    # its edge, and the polytope's own vertices among them: every point's
    # first facet, or none, must be found exactly.
    rng = np.random.default_rng(70)
    dirs = [[1, 0, 0], [-1, 0, 0], [0, 1, 0], [0, -1, 0], [0, 0, 1], [0, 0, -1]]
    dirs += [[sx, sy, sz] for sz in (1, -1) for sy in (1, -1) for sx in (1, -1)]
    E = np.array(dirs, np.float64)
    E /= np.linalg.norm(E, axis=1, keepdims=True)
    E += rng.normal(scale=2e-3, size=E.shape)  # general position: triangular facets
    E /= np.linalg.norm(E, axis=1, keepdims=True)
    E = (E + offset).astype(np.float32)
    _, faces = oracle.hull3d(E[:, 0], E[:, 1], E[:, 2])
    assert all(len(f) == 3 for f in faces) and len(faces) == 24
    E64 = E.astype(np.float64)
    c = np.float32(np.mean([E64[list(f)] for f in faces], axis=(0, 1))).astype(np.float64)
    dist, nrm = [], []
    for f in faces:
        a, b, d = E64[list(f)]
        n = np.cross(b - a, d - a)
        n /= np.linalg.norm(n)
        if np.dot(c - a, n) > 0:
            n = -n
        dist.append(np.dot(a - c, n))
        nrm.append(n)
    r = min(dist)
    assert r > 0.5
    ulp = float(np.spacing(np.float32(abs(offset) + 1.0)))
    Q = np.array([c + n * (dd + max(1e-5 * dd, 4 * ulp)) for n, dd in zip(nrm, dist)],
                 np.float32)
    # interior: a uniform ball to 0.98 r, and a shell around the test's
    # radius (inside the polytope: every point strictly below every facet)
    u = np.stack(w.uniform_ball(150_000, 71), axis=1).astype(np.float64)
    inner = c + 0.98 * r * u
    s = rng.normal(size=(30_000, 3))
    s /= np.linalg.norm(s, axis=1, keepdims=True)
    shell = c + s * r * (1.0 - rng.uniform(0.0, 2e-5, (30_000, 1)))
    filler = np.concatenate([inner, shell]).astype(np.float32)
    P = np.concatenate([filler[:70_000], E, filler[70_000:100_000], Q, filler[100_000:]])
    want = _oracle(P[:, 0], P[:, 1], P[:, 2])
    q0 = 70_000 + len(E) + 30_000
    assert set(range(q0, q0 + len(Q))) <= set(want[0])
    for pred in ("f32", "f64"):
        v, f, res = _gpu(qh, P[:, 0], P[:, 1], P[:, 2], pred=pred)
        assert res["status"] == 0
        assert (v, f) == (want[0], want[1]), pred
