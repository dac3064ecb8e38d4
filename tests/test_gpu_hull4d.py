"""GPU parity for the 4D hull (Section 4.3, higher dimensions): the extreme
points and the facet lists of the CUDA path (through the C ABI) equal the
oracle's, list for list, on seeded inputs: uniform in the 4-ball, near the
3-sphere (large hulls), Gaussian clouds, the tesseract with interior and
boundary points, the cross-polytope, lattice points on a 3-sphere,
duplicates, interleaved input, and degenerate and non-finite inputs."""
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


def _gpu(qh, x, y, z, ww, **kw):
    T = [torch.from_numpy(np.ascontiguousarray(c, dtype=np.float32)).cuda() for c in (x, y, z, ww)]
    (v, off, idx), res = qh.hull4d(*T, return_result=True, **kw)
    v, off, idx = v.cpu().numpy(), off.cpu().numpy(), idx.cpu().numpy()
    facets = [tuple(idx[off[i]:off[i + 1]].tolist()) for i in range(len(off) - 1)]
    return v.tolist(), facets, res


def _oracle(x, y, z, ww):
    v, f = oracle.hull4d(x, y, z, ww)
    return v.tolist(), [tuple(t.tolist()) for t in f]


@pytest.mark.parametrize("gen,n", [("ball", 1000), ("ball", 300_007), ("near", 20_000),
                                   ("near2", 60_001), ("gauss", 100_003), ("ball", 6),
                                   ("ball", 2049)])
def test_distributions_match_oracle(qh, gen, n):
    seed = 700 + n
    if gen == "ball":
        x, y, z, ww = w.uniform_ball_4d(n, seed)
    elif gen == "near":
        x, y, z, ww = w.near_sphere_4d(n, seed, 1e-3)
    elif gen == "near2":
        x, y, z, ww = w.near_sphere_4d(n, seed, 1e-2)
    else:
        x, y, z, ww = np.random.default_rng(seed).standard_normal((4, n)).astype(np.float32)
    gv, gf, res = _gpu(qh, x, y, z, ww)
    ov, of = _oracle(x, y, z, ww)
    assert res["status"] == 0
    assert gv == ov
    assert gf == of


def test_tesseract_interior_and_boundary(qh):
    rng = np.random.default_rng(71)
    corners = np.array([[i, j, k, l] for i in (-1, 1) for j in (-1, 1) for k in (-1, 1)
                        for l in (-1, 1)], np.float32)
    inner = rng.uniform(-0.99, 0.99, (20000, 4)).astype(np.float32)
    bnd = rng.uniform(-1, 1, (2000, 4)).astype(np.float32)
    for r in range(len(bnd)):
        fix = rng.choice(4, size=int(rng.integers(1, 4)), replace=False)
        bnd[r, fix] = rng.choice([-1.0, 1.0], len(fix))
    P = np.concatenate([bnd, inner, corners])
    P = P[rng.permutation(len(P))]
    gv, gf, _ = _gpu(qh, P[:, 0], P[:, 1], P[:, 2], P[:, 3])
    ov, of = _oracle(P[:, 0], P[:, 1], P[:, 2], P[:, 3])
    assert len(gv) == 16 and gv == ov
    assert len(gf) == 8 and gf == of


def test_cross_polytope_lattice_sphere_duplicates(qh):
    rng = np.random.default_rng(72)
    tips = np.vstack([np.eye(4), -np.eye(4)]).astype(np.float32)
    P = np.concatenate([rng.uniform(-0.2, 0.2, (3000, 4)).astype(np.float32), tips, tips])
    gv, gf, _ = _gpu(qh, *P.T)
    assert (gv, gf) == _oracle(*P.T)
    assert len(gf) == 16
    lat = np.array([(a, b, c, d) for a in range(-5, 6) for b in range(-5, 6)
                    for c in range(-5, 6) for d in range(-5, 6)
                    if a * a + b * b + c * c + d * d == 27], np.float32)
    inner = (2.5 * np.stack(w.uniform_ball_4d(5000, 73), axis=1)).astype(np.float32)
    Q = np.concatenate([inner, lat])
    gv, gf, _ = _gpu(qh, *Q.T)
    ov, of = _oracle(*Q.T)
    assert gv == ov and gv == list(range(5000, 5000 + len(lat)))
    assert sorted(gf) == sorted(of)  # facets of more than eight vertices: order on the first eight


def test_interleaved_input(qh):
    x, y, z, ww = w.uniform_ball_4d(50_001, 74)
    P = torch.from_numpy(np.stack([x, y, z, ww], axis=1).copy()).cuda()
    v, off, idx = qh.hull4d(P)
    ov, of = _oracle(x, y, z, ww)
    assert v.cpu().numpy().tolist() == ov
    o, ix = off.cpu().numpy(), idx.cpu().numpy()
    assert [tuple(ix[o[i]:o[i + 1]].tolist()) for i in range(len(o) - 1)] == of


def test_degenerate_and_nonfinite(qh):
    rng = np.random.default_rng(75)
    p = rng.random((3, 500)).astype(np.float32)
    with pytest.raises(qh.QHError) as ei:  # all points in the hyperplane w = 0.25
        _gpu(qh, p[0], p[1], p[2], np.full(500, 0.25, np.float32))
    assert ei.value.status == 3
    with pytest.raises(qh.QHError) as ei:
        _gpu(qh, *rng.random((4, 4)).astype(np.float32))
    assert ei.value.status == 3
    bad = rng.random((4, 1000)).astype(np.float32)
    bad[3, 777] = np.inf
    with pytest.raises(qh.QHError) as ei:
        _gpu(qh, *bad)
    assert ei.value.status == 2
    gv, gf, res = _gpu(qh, *(np.zeros(0, np.float32) for _ in range(4)))
    assert gv == [] and gf == [] and res["status"] == 0


@pytest.mark.parametrize("scale", [1e13, 1e-20])
def test_filter_overflow_and_underflow_scales(qh, scale):
    # coordinates whose FP32 filter products overflow (1e13) or underflow
    # (1e-20): the exact path decides, the hull is the oracle's
    x, y, z, ww = w.uniform_ball_4d(20_000, 76)
    s = np.float32(scale)
    P = [(c * s).astype(np.float32) for c in (x, y, z, ww)]
    gv, gf, res = _gpu(qh, *P)
    assert res["status"] == 0
    assert (gv, gf) == _oracle(*P)


def test_every_point_twice_and_signed_zeros(qh):
    # each point also at a higher index, some of the copies with -0.0 for
    # 0.0: every vertex is reported by its lowest index, as in the oracle
    rng = np.random.default_rng(77)
    pts = np.stack(w.uniform_ball_4d(4_000, 78), axis=1).astype(np.float32)
    pts[rng.integers(0, 4_000, 200), rng.integers(0, 4, 200)] = np.float32(0.0)
    twin = pts.copy()
    twin[twin == 0] = np.float32(-0.0)
    P = np.concatenate([pts, twin])
    P = np.concatenate([P, pts[rng.permutation(4_000)]])
    gv, gf, res = _gpu(qh, *P.T)
    assert res["status"] == 0
    assert (gv, gf) == _oracle(*P.T)
