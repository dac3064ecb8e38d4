"""Pins for the oracle's hull measures and gradients: closed forms (unit
square, regular polygon, tetrahedron, octahedron) and central finite
differences (h = 1e-3) of the measure of the recomputed hull."""
import math

import numpy as np
import pytest

import oracle
from oracle import measures as M


def test_unit_square_closed_form():
    x = np.array([0, 1, 1, 0, 0.5], np.float32)
    y = np.array([0, 0, 1, 1, 0.5], np.float32)
    hull = oracle.hull2d(x, y).tolist()
    assert hull == [0, 1, 2, 3]
    per, area = M.measures2d(x, y, hull)
    assert per == 4.0 and area == 1.0
    gx, gy = M.grad2d(x, y, hull, 1.0, 0.0)
    assert (gx[0], gy[0]) == (-1.0, -1.0) and (gx[2], gy[2]) == (1.0, 1.0)
    gx, gy = M.grad2d(x, y, hull, 0.0, 1.0)
    assert (gx[0], gy[0]) == (-0.5, -0.5) and (gx[1], gy[1]) == (0.5, -0.5)
    assert gx[4] == 0.0 and gy[4] == 0.0  # interior point


@pytest.mark.parametrize("m", [3, 5, 12, 40])
def test_regular_polygon_radial_derivatives(m):
    r = 0.75
    th = 2 * np.pi * np.arange(m) / m
    x, y = r * np.cos(th), r * np.sin(th)
    hull = list(range(m))
    per, area = M.measures2d(x, y, hull)
    assert per == pytest.approx(2 * m * r * math.sin(math.pi / m), rel=1e-13)
    assert area == pytest.approx(0.5 * m * r * r * math.sin(2 * math.pi / m), rel=1e-13)
    # scaling every vertex radially: sum of gradient . (p / r) = d(measure)/dr
    for wp, wa, want in ((1, 0, 2 * m * math.sin(math.pi / m)),
                         (0, 1, m * r * math.sin(2 * math.pi / m))):
        gx, gy = M.grad2d(x, y, hull, wp, wa)
        assert float(np.sum(gx * x + gy * y) / r) == pytest.approx(want, rel=1e-12)


def test_tetrahedron_and_octahedron_closed_forms():
    P = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], np.float32)
    v, faces = oracle.hull3d(P[:, 0], P[:, 1], P[:, 2])
    area, vol = M.measures3d(P[:, 0], P[:, 1], P[:, 2], faces)
    assert vol == pytest.approx(1 / 6, rel=1e-15)
    assert area == pytest.approx(1.5 + math.sqrt(3) / 2, rel=1e-15)
    g = M.grad3d(P[:, 0], P[:, 1], P[:, 2], faces, 0.0, 1.0)
    assert np.allclose(g[3], [0, 0, 1 / 6], rtol=0, atol=1e-15)
    assert np.allclose(g[0], [-1 / 6, -1 / 6, -1 / 6], rtol=0, atol=1e-15)
    r = 0.5
    O = np.array([[r, 0, 0], [-r, 0, 0], [0, r, 0], [0, -r, 0], [0, 0, r], [0, 0, -r]], np.float32)
    v, faces = oracle.hull3d(O[:, 0], O[:, 1], O[:, 2])
    assert len(faces) == 8
    area, vol = M.measures3d(O[:, 0], O[:, 1], O[:, 2], faces)
    assert vol == pytest.approx(4 / 3 * r ** 3, rel=1e-14)
    assert area == pytest.approx(4 * math.sqrt(3) * r * r, rel=1e-14)
    for wa, wv, want in ((1, 0, 8 * math.sqrt(3) * r), (0, 1, 4 * r * r)):
        g = M.grad3d(O[:, 0], O[:, 1], O[:, 2], faces, wa, wv)
        assert float(np.sum(g * O) / r) == pytest.approx(want, rel=1e-13)


def _fd_check(evaluate, grad, coords, idx_list, h=1e-3):
    """Central differences of evaluate() over the listed coordinates; the
    perturbed value is rounded to float32 and the quotient uses the actual
    step.  Coordinates whose perturbation changes the hull are skipped."""
    base_struct = evaluate(coords)[1]
    num, ana = [], []
    for (k, i) in idx_list:
        c0 = coords[k][i]
        up, dn = np.float32(c0 + h), np.float32(c0 - h)
        coords[k][i] = up
        fu, su = evaluate(coords)
        coords[k][i] = dn
        fd_, sd = evaluate(coords)
        coords[k][i] = c0
        if su != base_struct or sd != base_struct:
            continue
        num.append((fu - fd_) / (float(up) - float(dn)))
        ana.append(grad[k][i])
    num, ana = np.array(num), np.array(ana)
    assert len(num) >= 4
    err = np.linalg.norm(num - ana) / np.linalg.norm(ana)
    assert err < 1e-4, err


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_grad2d_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    n = 60
    rad, th = np.sqrt(rng.random(n)), 2 * np.pi * rng.random(n)
    coords = [(rad * np.cos(th)).astype(np.float32), (rad * np.sin(th)).astype(np.float32)]
    wp, wa = rng.uniform(0.5, 2.0, 2)

    def evaluate(c):
        hull = oracle.hull2d(c[0], c[1]).tolist()
        p, a = M.measures2d(c[0], c[1], hull)
        return wp * p + wa * a, tuple(hull)

    hull = oracle.hull2d(*coords).tolist()
    gx, gy = M.grad2d(coords[0], coords[1], hull, wp, wa)
    idx = [(k, i) for i in hull for k in (0, 1)] + [(0, i) for i in range(n) if i not in hull][:5]
    _fd_check(evaluate, [gx, gy], coords, idx)


@pytest.mark.parametrize("seed", [4, 5])
def test_grad3d_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    n = 40
    g = rng.standard_normal((3, n))
    g *= rng.random(n) ** (1 / 3) / np.linalg.norm(g, axis=0)
    coords = [c.astype(np.float32) for c in g]
    wa, wv = rng.uniform(0.5, 2.0, 2)

    def evaluate(c):
        v, faces = oracle.hull3d(c[0], c[1], c[2])
        a, vol = M.measures3d(c[0], c[1], c[2], faces)
        return wa * a + wv * vol, tuple(tuple(f.tolist()) for f in faces)

    v, faces = oracle.hull3d(*coords)
    G = M.grad3d(coords[0], coords[1], coords[2], faces, wa, wv)
    idx = [(k, i) for i in v.tolist() for k in (0, 1, 2)]
    _fd_check(evaluate, [G[:, 0], G[:, 1], G[:, 2]], coords, idx)
