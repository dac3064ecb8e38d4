"""GPU differentiable hulls: the measures (2D perimeter and area, 3D surface
area and volume) equal the oracle's FP64 measures of the oracle's hull, the
hand-written backward kernels' gradients equal the oracle's FP64 gradients
(relative error below 1e-4, exactly zero off the hull), and central finite
differences (h = 1e-3) of the GPU measures agree with the GPU gradients."""
import numpy as np
import pytest
import torch

import oracle
from oracle import measures as M
from paper_1201_2936_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qh():
    from paper_1201_2936_gb300 import build
    build.build()
    oracle.build()
    import paper_1201_2936_gb300 as q
    return q


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _check2d(qh, x, y, off, weights, full_grad=True):
    P = torch.from_numpy(np.stack([x, y])).cuda().requires_grad_(True)
    O = torch.from_numpy(off).cuda()
    meas = qh.hull_measures_2d(P, O)
    W = torch.from_numpy(weights).cuda()
    (meas * W).sum().backward()
    m = meas.detach().cpu().numpy()
    g = P.grad.cpu().numpy()
    for c in range(len(off) - 1):
        a, b = int(off[c]), int(off[c + 1])
        hull = oracle.hull2d(x[a:b], y[a:b]).tolist()
        per, area = M.measures2d(x[a:b], y[a:b], hull)
        assert m[c, 0] == pytest.approx(per, rel=1e-12)
        assert m[c, 1] == pytest.approx(area, rel=1e-12)
        if full_grad:
            gx, gy = M.grad2d(x[a:b], y[a:b], hull, weights[c, 0], weights[c, 1])
            want = np.stack([gx, gy])
            assert _rel(g[:, a:b], want) < 1e-4, c
            off_hull = np.ones(b - a, bool)
            off_hull[hull] = False
            assert not np.any(g[:, a:b][:, off_hull])
    return P, O, g


def _check3d(qh, x, y, z, off, weights):
    P = torch.from_numpy(np.stack([x, y, z])).cuda().requires_grad_(True)
    O = torch.from_numpy(off).cuda()
    meas = qh.hull_measures_3d(P, O)
    W = torch.from_numpy(weights).cuda()
    (meas * W).sum().backward()
    m = meas.detach().cpu().numpy()
    g = P.grad.cpu().numpy()
    for c in range(len(off) - 1):
        a, b = int(off[c]), int(off[c + 1])
        v, faces = oracle.hull3d(x[a:b], y[a:b], z[a:b])
        area, vol = M.measures3d(x[a:b], y[a:b], z[a:b], faces)
        assert m[c, 0] == pytest.approx(area, rel=1e-12)
        assert m[c, 1] == pytest.approx(vol, rel=1e-12)
        G = M.grad3d(x[a:b], y[a:b], z[a:b], faces, weights[c, 0], weights[c, 1])
        assert _rel(g[:, a:b].T, G) < 1e-4, c
        off_hull = np.ones(b - a, bool)
        off_hull[v] = False
        assert not np.any(g[:, a:b][:, off_hull])
    return P, O, g


def test_2d_small_batch_and_finite_differences(qh):
    x, y, off = w.batched_disk_2d(16, 512, 21)
    rng = np.random.default_rng(0)
    wts = rng.uniform(0.5, 2.0, (16, 2))
    P, O, g = _check2d(qh, x, y, off, wts)
    # central differences of the GPU measures against the GPU gradient
    W = torch.from_numpy(wts).cuda()
    base = P.detach().clone()

    def loss(Q):
        with torch.no_grad():
            return float((qh.hull_measures_2d(Q, O) * W).sum())

    hull0 = oracle.hull2d(x[:512], y[:512]).tolist()
    num, ana = [], []
    for i in hull0[:8]:
        for k in (0, 1):
            Q = base.clone()
            up = np.float32(base[k, i].item() + 1e-3)
            dn = np.float32(base[k, i].item() - 1e-3)
            Q[k, i] = float(up)
            fu = loss(Q)
            Q[k, i] = float(dn)
            fd_ = loss(Q)
            num.append((fu - fd_) / (float(up) - float(dn)))
            ana.append(g[k, i])
    assert _rel(np.array(num), np.array(ana)) < 1e-4


def test_3d_small_batch(qh):
    x, y, z, off = w.batched_ball_3d(8, 2048, 22)
    rng = np.random.default_rng(1)
    _check3d(qh, x, y, z, off, rng.uniform(0.5, 2.0, (8, 2)))


def test_full_size_2d(qh):
    # 1024 clouds x 4096 points in the disk, loss = sum of perimeters + areas
    x, y, off = w.batched_disk_2d(1024, 4096, w.SEED_BASE + 4)
    _check2d(qh, x, y, off, np.ones((1024, 2)))


def test_full_size_3d(qh):
    # 256 clouds x 16384 points in the ball, loss = sum of volumes + areas
    x, y, z, off = w.batched_ball_3d(256, 16384, w.SEED_BASE + 5)
    _check3d(qh, x, y, z, off, np.ones((256, 2)))
