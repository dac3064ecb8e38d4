"""GPU parity for the 2D hull: the CUDA path (through the C ABI) against the
oracle, index for index, on seeded inputs: several tiles with ragged tails,
the paper's distributions, degenerate inputs, both predicate modes and both
loop drivers."""
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


def _gpu(qh, x, y, **kw):
    X = torch.from_numpy(np.asarray(x, np.float32)).cuda()
    Y = torch.from_numpy(np.asarray(y, np.float32)).cuda()
    idx, res = qh.hull2d(X, Y, return_result=True, **kw)
    return idx.cpu().numpy(), res


MODES = [dict(pred="f32", loop="persistent"), dict(pred="f64", loop="host"),
         dict(pred="f32", loop="host"), dict(pred="f64", loop="persistent")]


@pytest.mark.parametrize("mode", MODES, ids=lambda m: f"{m['pred']}-{m['loop']}")
def test_square_100k_matches_oracle(qh, mode):
    x, y = w.uniform_square(w.N_SMALL_2D, w.SEED_BASE + 0)
    got, res = _gpu(qh, x, y, **mode)
    want = oracle.hull2d(x, y)
    assert got.tolist() == want.tolist()
    assert res["status"] == 0 and res["count"] == len(want)


@pytest.mark.parametrize("gen,n", [("disk", 300_001), ("circle", 250_037), ("square", 4097),
                                   ("gauss", 1_000_003), ("circle", 2049), ("disk", 2047)])
def test_distributions_match_oracle(qh, gen, n):
    seed = 77 + n
    if gen == "disk":
        x, y = w.uniform_disk(n, seed)
    elif gen == "circle":
        x, y = w.circle_jitter(n, seed, 1e-4)
    elif gen == "square":
        x, y = w.uniform_square(n, seed)
    else:
        r = np.random.default_rng(seed)
        x, y = r.normal(size=(2, n)).astype(np.float32)
    want = oracle.hull2d(x, y)
    for mode in MODES[:2]:
        got, res = _gpu(qh, x, y, **mode)
        assert got.tolist() == want.tolist(), mode


def test_tiny_and_degenerate(qh):
    cases = [
        ([], []),
        ([1.5], [2.5]),
        ([1, 1, 1, 1], [2, 2, 2, 2]),
        ([0, 1], [0, 1]),
        ([1, 0], [1, 0]),
        ([2, 0, 1, 3], [2, 0, 1, 3]),               # collinear
        ([0, 1, 0, 1, 1, 0], [0, 0, 1, 1, 0, 0]),   # duplicates of vertices
        ([0.0, -0.0, 1.0, 0.0], [0.0, 0.0, 0.0, 1.0]),
        ([0, 2, 1, 1, 1], [0, 0, 1, 1, -1]),
    ]
    rng = np.random.default_rng(3)
    for _ in range(40):
        n = int(rng.integers(1, 60))
        cases.append((rng.integers(0, 4, n).tolist(), rng.integers(0, 4, n).tolist()))
    for x, y in cases:
        x = np.asarray(x, np.float32)
        y = np.asarray(y, np.float32)
        want = oracle.hull2d(x, y)
        for mode in MODES:
            got, res = _gpu(qh, x, y, **mode)
            assert got.tolist() == want.tolist(), (x, y, mode)


def test_integer_grid_many_ties(qh):
    # lattice points: many exact distance ties, collinear runs on every side
    rng = np.random.default_rng(5)
    x = rng.integers(-300, 301, 400_000).astype(np.float32)
    y = rng.integers(-200, 201, 400_000).astype(np.float32)
    want = oracle.hull2d(x, y)
    for mode in MODES[:2]:
        got, res = _gpu(qh, x, y, **mode)
        assert got.tolist() == want.tolist()
        assert res["exact_argmax"] > 0


def test_integer_circle_all_vertices(qh):
    r = 5 ** 4  # x^2 + y^2 = 625^2: every lattice point is a hull vertex
    pts = set()
    for i in range(-r, r + 1):
        j2 = r * r - i * i
        j = int(np.sqrt(j2))
        while j * j > j2:
            j -= 1
        while (j + 1) ** 2 <= j2:
            j += 1
        if j * j == j2:
            pts.add((i, j))
            pts.add((i, -j))
    pts = np.array(sorted(pts), np.float32)
    rng = np.random.default_rng(2)
    inner = rng.uniform(-400, 400, (100_000, 2)).astype(np.float32)
    P = np.concatenate([inner, pts])[rng.permutation(len(inner) + len(pts))]
    want = oracle.hull2d(P[:, 0], P[:, 1])
    assert len(want) == len(pts)
    got, _ = _gpu(qh, P[:, 0], P[:, 1])
    assert got.tolist() == want.tolist()


def test_interleaved_and_soa_layouts(qh):
    x, y = w.uniform_disk(100_003, 12)
    want = oracle.hull2d(x, y)
    P = torch.from_numpy(np.stack([x, y], 1)).cuda()       # [n, 2], stride 2
    assert qh.hull2d(P).cpu().numpy().tolist() == want.tolist()
    Q = torch.from_numpy(np.stack([x, y], 0)).cuda()       # [2, n]
    assert qh.hull2d(Q).cpu().numpy().tolist() == want.tolist()


def test_nonfinite_is_reported(qh):
    x = np.array([0, 1, np.nan, 3], np.float32)
    y = np.array([0, 1, 2, 3], np.float32)
    for mode in MODES[:2]:
        with pytest.raises(qh.QHError) as ei:
            _gpu(qh, x, y, **mode)
        assert ei.value.status == 2


def test_repeat_calls_reuse_workspace(qh):
    x, y = w.circle_jitter(500_000, 3, 1e-4)
    want = oracle.hull2d(x, y)
    ws = qh.Workspace()
    for _ in range(3):
        X, Y = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        assert qh.hull2d(X, Y, workspace=ws).cpu().numpy().tolist() == want.tolist()


@pytest.mark.parametrize("ctas", [1, 2, 3])
def test_capped_grid_long_runs(qh, ctas):
    # few CTAs: each one's run of tiles is longer than the tile map it stages
    for x, y in (w.uniform_disk(1_000_003, 5), w.circle_jitter(700_001, 6, 1e-4)):
        want = oracle.hull2d(x, y)
        X, Y = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        got = qh.hull2d(X, Y, opts=qh.make_opts("f32", max_ctas=ctas))
        assert got.cpu().numpy().tolist() == want.tolist(), ctas


def test_unaligned_inputs(qh):
    # coordinates that start off a 16-byte boundary (no bulk copies of the
    # caller's arrays in the first pass)
    x, y = w.uniform_disk(200_001, 8)
    want = oracle.hull2d(x[1:], y[1:])
    X = torch.from_numpy(x).cuda()[1:]
    Y = torch.from_numpy(y).cuda()[1:]
    assert qh.hull2d(X, Y).cpu().numpy().tolist() == want.tolist()


@pytest.mark.parametrize("cloud", ["square", "disk", "circle1e-4"])
def test_full_size_bench_clouds(qh, cloud):
    # the 2D benchmark workload at full size (16M points per cloud), in the
    # launch configuration the benchmark times (persistent kernel, FP32 filter)
    s = w.SEED_BASE + 1
    if cloud == "square":
        x, y = w.uniform_square(w.N_LARGE_2D, s)
    elif cloud == "disk":
        x, y = w.uniform_disk(w.N_LARGE_2D, s + 10)
    else:
        x, y = w.circle_jitter(w.N_LARGE_2D, s + 20, 1e-4)
    want = oracle.hull2d(x, y)
    P = torch.from_numpy(np.stack([x, y])).cuda()
    got = qh.hull2d(P)
    assert got.cpu().numpy().tolist() == want.tolist()


@pytest.mark.parametrize("loop", ["persistent", "host"])
def test_hull_larger_than_block_output(qh, loop):
    # every point of y = x^2 (exact in float32 for |x| < 4096) is a vertex:
    # 8191 hull vertices, more than one block ranks in shared memory, plus
    # interior points, shuffled
    r = np.random.default_rng(11)
    i = np.arange(-4095, 4096, dtype=np.float64)
    cx, cy = i, i * i
    # interior: strictly above the parabola and below the chord y = 4095^2
    top = 4095.0 * 4095.0
    ix = np.round(r.uniform(-4000, 4000, 50_000))
    iy = np.round(ix * ix + 1 + r.uniform(0, 1, ix.size) * (top - 2 - ix * ix))
    x = np.concatenate([cx, ix]).astype(np.float32)
    y = np.concatenate([cy, iy]).astype(np.float32)
    p = r.permutation(x.size)
    x, y = x[p], y[p]
    want = oracle.hull2d(x, y)
    assert len(want) == 8191
    # (the synchronous entry point finishes such hulls with the large-hull
    # output step)
    got, res = _gpu(qh, x, y, pred="f32", loop=loop)
    assert res["status"] == 0
    assert got.tolist() == want.tolist()


def test_many_vertices_on_circle(qh):
    # 300k float32 points on the unit circle: thousands of exact extreme points
    r = np.random.default_rng(12)
    t = r.uniform(0, 2 * np.pi, 300_000)
    x, y = np.cos(t).astype(np.float32), np.sin(t).astype(np.float32)
    want = oracle.hull2d(x, y)
    assert len(want) > 4096
    got, res = _gpu(qh, x, y, pred="f32", loop="persistent")
    assert res["status"] == 0
    assert got.tolist() == want.tolist()


@pytest.mark.parametrize("scale", [1e-20, 1e-30, 1e20])
def test_filter_scales_2d(qh, scale):
    x, y = w.uniform_disk(200_000, 67)
    s = np.float32(scale)
    X, Y = (x * s).astype(np.float32), (y * s).astype(np.float32)
    want = oracle.hull2d(X, Y).tolist()
    for loop in ("persistent", "host"):
        got = qh.hull2d(torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda(), loop=loop)
        assert got.cpu().numpy().tolist() == want, loop


def test_unaligned_inputs_take_the_plain_load_path(qh):
    # bases that are not 16-byte aligned (a view one float in, an interleaved
    # view one point in): the first pass reads them without bulk copies
    x, y = w.uniform_disk(300_001, 68)
    X = torch.from_numpy(np.concatenate([[0.0], x]).astype(np.float32)).cuda()[1:]
    Y = torch.from_numpy(np.concatenate([[0.0], y]).astype(np.float32)).cuda()[1:]
    assert X.data_ptr() % 16 != 0
    want = oracle.hull2d(x, y).tolist()
    assert qh.hull2d(X, Y).cpu().numpy().tolist() == want
    P = torch.from_numpy(np.stack([np.concatenate([[0.0], x]), np.concatenate([[0.0], y])],
                                  axis=1).astype(np.float32)).cuda()[1:]
    assert P.data_ptr() % 16 != 0
    assert qh.hull2d(P).cpu().numpy().tolist() == want
    got = qh.hull2d_multi([(X, Y), P, (X[:1000], Y[:1000])])
    assert got[0].cpu().numpy().tolist() == want
    assert got[1].cpu().numpy().tolist() == want
    assert got[2].cpu().numpy().tolist() == oracle.hull2d(x[:1000], y[:1000]).tolist()
