"""GPU parity for several 2D clouds in one persistent launch: each cloud's
hull (through the C ABI) against the oracle's hull of that cloud alone,
index for index, on seeded inputs of mixed distributions and sizes, with the
degenerate clouds (empty, one point, identical points, collinear points,
non-finite) beside normal ones."""
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


def _dev(x, y):
    return (torch.from_numpy(np.asarray(x, np.float32)).cuda(),
            torch.from_numpy(np.asarray(y, np.float32)).cuda())


def _check(qh, clouds, pred="f32"):
    got, res = qh.hull2d_multi([_dev(x, y) for x, y in clouds], pred=pred, return_results=True)
    for c, (x, y) in enumerate(clouds):
        if len(x) and not (np.isfinite(x).all() and np.isfinite(y).all()):
            assert res[c]["status"] == 2, c  # QH_ERR_NONFINITE
            continue
        assert res[c]["status"] == 0, (c, res[c])
        want = oracle.hull2d(np.asarray(x, np.float32), np.asarray(y, np.float32)) if len(x) else []
        assert got[c].cpu().numpy().tolist() == list(want), c


@pytest.mark.parametrize("pred", ["f32", "f64"])
def test_mixed_clouds_match_oracle(qh, pred):
    r = np.random.default_rng(3)
    g = r.normal(size=(2, 50_001)).astype(np.float32)
    clouds = [w.uniform_square(100_000, 11), w.uniform_disk(300_001, 12),
              w.circle_jitter(250_037, 13, 1e-4), (g[0], g[1]), w.uniform_disk(2047, 14),
              w.uniform_square(5, 15)]
    _check(qh, clouds, pred)


def test_degenerate_clouds_beside_normal_ones(qh):
    x, y = w.uniform_disk(70_001, 21)
    bad = np.array([0.5, np.nan, 0.25], np.float32)
    clouds = [
        (x, y),
        (np.zeros(0, np.float32), np.zeros(0, np.float32)),   # empty
        (np.array([0.3], np.float32), np.array([0.7], np.float32)),  # one point
        (np.full(1000, 2.5, np.float32), np.full(1000, -1.0, np.float32)),  # identical
        (np.arange(100, dtype=np.float32), 2 * np.arange(100, dtype=np.float32)),  # collinear
        (bad, np.array([0.1, 0.2, 0.3], np.float32)),  # non-finite
        w.circle_jitter(9_999, 22, 1e-4),
        w.uniform_square(33_333, 23),
    ]
    _check(qh, clouds)


def test_single_cloud_equals_hull2d(qh):
    x, y = w.circle_jitter(400_000, 31, 1e-4)
    X, Y = _dev(x, y)
    one = qh.hull2d_multi([(X, Y)])[0]
    assert one.cpu().numpy().tolist() == qh.hull2d(X, Y).cpu().numpy().tolist()


def test_layouts_and_large_hull(qh):
    # an interleaved [n, 2] cloud, an unaligned one and a hull with 8191
    # vertices (more hull slots than one block ranks in shared memory)
    i = np.arange(-4095, 4096, dtype=np.float64)
    px, py = i.astype(np.float32), (i * i).astype(np.float32)
    x1, y1 = w.uniform_disk(60_001, 41)
    x2, y2 = w.uniform_square(80_000, 42)
    P1 = torch.from_numpy(np.stack([x1, y1], 1).copy()).cuda()
    X2 = torch.from_numpy(np.concatenate([[0.0], x2]).astype(np.float32)).cuda()[1:]
    Y2 = torch.from_numpy(np.concatenate([[0.0], y2]).astype(np.float32)).cuda()[1:]
    got = qh.hull2d_multi([_dev(px, py), P1, (X2, Y2)])
    assert got[0].cpu().numpy().tolist() == oracle.hull2d(px, py).tolist()
    assert got[1].cpu().numpy().tolist() == oracle.hull2d(x1, y1).tolist()
    assert got[2].cpu().numpy().tolist() == oracle.hull2d(x2, y2).tolist()


def test_full_size_bench_clouds_in_one_launch(qh):
    # the 2D benchmark workload (three 16M-point clouds) in the launch the
    # benchmark times
    s = w.SEED_BASE + 1
    clouds = [w.uniform_square(w.N_LARGE_2D, s), w.uniform_disk(w.N_LARGE_2D, s + 10),
              w.circle_jitter(w.N_LARGE_2D, s + 20, 1e-4)]
    got = qh.hull2d_multi([torch.from_numpy(np.stack([x, y])).cuda() for x, y in clouds])
    for c, (x, y) in enumerate(clouds):
        assert got[c].cpu().numpy().tolist() == oracle.hull2d(x, y).tolist(), c


def _tie_and_overflow_clouds():
    r = np.random.default_rng(51)
    # integer parabola y = x^2 (every point a hull vertex) with interior
    # points above it: the farthest points of a segment whose ends are
    # (a, a^2), (b, b^2) with a + b odd tie exactly, (i - a)(b - i) at
    # i = (a + b -+ 1) / 2; all coordinates are exact in float32
    i = np.arange(-1500, 1501)
    ix = r.integers(-1400, 1401, 30_000)
    iy = ix * ix + 1 + r.integers(0, 10_000, 30_000)
    x = np.concatenate([i, ix]).astype(np.float32)
    y = np.concatenate([i * i, np.minimum(iy, 1500 * 1500 - 1)]).astype(np.float32)
    p = r.permutation(len(x))
    parabola = (x[p], y[p])
    # hull vertices of a disk repeated at higher and lower indices
    dx, dy = w.uniform_disk(50_000, 52)
    hv = oracle.hull2d(dx, dy)[:12]
    dup = (np.concatenate([dx[hv], dx, dx[hv]]).astype(np.float32),
           np.concatenate([dy[hv], dy, dy[hv]]).astype(np.float32))
    # coordinates near 1e37: the FP32 filter overflows, the exact path decides
    hx, hy = w.uniform_disk(20_000, 53)
    huge = ((hx * np.float32(1e37)).astype(np.float32), (hy * np.float32(1e37)).astype(np.float32))
    # a shuffled integer grid: collinear points on every hull edge, equal
    # distances everywhere
    gx, gy = np.meshgrid(np.arange(300, dtype=np.float32), np.arange(300, dtype=np.float32))
    q = r.permutation(300 * 300)
    grid = (gx.ravel()[q].copy(), gy.ravel()[q].copy())
    return [parabola, dup, huge, grid]


@pytest.mark.parametrize("pred", ["f32", "f64"])
def test_exact_ties_and_filter_overflow(qh, pred):
    clouds = _tie_and_overflow_clouds()
    _check(qh, clouds, pred)
    for c, (x, y) in enumerate(clouds):
        X, Y = _dev(x, y)
        got = qh.hull2d(X, Y, pred=pred)
        assert got.cpu().numpy().tolist() == oracle.hull2d(x, y).tolist(), c


@pytest.mark.parametrize("ctas", [1, 2, 3])
def test_capped_grid_long_runs(qh, ctas):
    # few CTAs: each one's run of tiles is longer than the tile map it stages,
    # so the producer searches the starts of straddling tiles' segments itself
    clouds = [w.uniform_disk(700_001, 71), w.circle_jitter(500_003, 72, 1e-4),
              w.uniform_square(300_007, 73)]
    got = qh.hull2d_multi([_dev(x, y) for x, y in clouds], opts=qh.make_opts("f32", max_ctas=ctas))
    for c, (x, y) in enumerate(clouds):
        assert got[c].cpu().numpy().tolist() == oracle.hull2d(x, y).tolist(), (ctas, c)


def test_duplicated_hull_vertices_large(qh):
    # every hull vertex of a 4M-point disk repeated at a higher index: each
    # segment's farthest point ties, so no apex is certified and the large
    # early segments go through the exact argmax split over many CTAs; the
    # hull keeps the lower index of every pair
    x, y = w.uniform_disk(4_000_000, 81)
    h = oracle.hull2d(x, y)
    xd = np.concatenate([x, x[h]]).astype(np.float32)
    yd = np.concatenate([y, y[h]]).astype(np.float32)
    sq = w.uniform_square(1_000_000, 82)
    got, res = qh.hull2d_multi([_dev(xd, yd), _dev(*sq)], return_results=True)
    assert got[0].cpu().numpy().tolist() == oracle.hull2d(xd, yd).tolist() == h.tolist()
    assert got[1].cpu().numpy().tolist() == oracle.hull2d(*sq).tolist()
    assert res[0]["exact_argmax"] > 0
