"""The multi-rank hull's default path on one GPU rank: the library's hull of
the shard, then of the gathered candidates, equals the direct hull."""
import numpy as np
import pytest
import torch

import oracle
from paper_1201_2936_gb300 import workloads as w

pytestmark = pytest.mark.gpu


def test_single_rank_sharded_hull_matches():
    from paper_1201_2936_gb300 import build, shard
    build.build()
    oracle.build()
    x, y = w.uniform_disk(200_000, 91)
    final, _ = shard.sharded_hull([torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()])
    assert final.cpu().numpy().tolist() == oracle.hull2d(x, y).tolist()
    x, y, z = w.uniform_ball(100_000, 92)
    final, _ = shard.sharded_hull([torch.from_numpy(c).cuda() for c in (x, y, z)])
    assert final.cpu().numpy().tolist() == oracle.hull3d(x, y, z)[0].tolist()


def _simulated(clouds, world, cap=16384, exchange_fail=None):
    """The ShardedHull2D device steps for `world` ranks in one process: each
    virtual rank's block written into its slot of the gathered buffer (what
    the all-gather produces), then the merge."""
    from paper_1201_2936_gb300 import shard
    T = [torch.from_numpy(np.stack(c)).cuda() for c in clouds]
    ranges = [[shard.shard_range(t.shape[1], r, world) for t in T] for r in range(world)]
    views = [[t[:, lo:hi] for t, (lo, hi) in zip(T, ranges[r])] for r in range(world)]
    sh = shard.ShardedHull2D([(v[0].contiguous(), v[1].contiguous()) for v in views[0]],
                             [lo for lo, _ in ranges[0]], world, 0, cap=cap)
    g = sh.gathered.view(world, -1)
    for r in range(world):
        sh.local_block([(v[0].contiguous(), v[1].contiguous()) for v in views[r]],
                       [lo for lo, _ in ranges[r]], g[r])
    sh.merge()
    return sh.results()


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_sharded_2d_device_steps_match_oracle(world):
    from paper_1201_2936_gb300 import build
    build.build()
    oracle.build()
    x, y = w.uniform_disk(300_001, 93)
    # duplicates of hull vertices in later shards, and an exact tie
    x = np.concatenate([x, x[:200], np.float32([2.0, 2.0])]).astype(np.float32)
    y = np.concatenate([y, y[:200], np.float32([0.5, 0.5])]).astype(np.float32)
    clouds = [(x, y), w.uniform_square(100_000, 94), w.circle_jitter(50_000, 95)]
    hulls, st = _simulated(clouds, world)
    assert st == [0, 0, 0]
    for h, (cx, cy) in zip(hulls, clouds):
        assert h.cpu().numpy().tolist() == oracle.hull2d(cx, cy).tolist()


def test_sharded_2d_reports_capacity_and_failed_shards():
    from paper_1201_2936_gb300 import build
    build.build()
    x, y = w.circle_jitter(40_000, 96)  # shard hulls above a cap of 16
    _, st = _simulated([(x, y)], 2, cap=16)
    assert st == [5]
    x2, y2 = w.uniform_disk(10_000, 97)
    x2[9_000] = np.nan  # in the second shard only
    _, st = _simulated([(x2, y2)], 2)
    assert st == [2]


def test_single_rank_sharded_hull3d_faces_match():
    from paper_1201_2936_gb300 import build, shard
    build.build()
    oracle.build()
    x, y, z = w.uniform_ball(80_000, 98)
    v, off, idx = shard.sharded_hull3d([torch.from_numpy(c).cuda() for c in (x, y, z)])
    wv, wf = oracle.hull3d(x, y, z)
    off, idx = off.cpu().numpy(), idx.cpu().numpy()
    assert v.cpu().numpy().tolist() == wv.tolist()
    assert [idx[off[i]:off[i + 1]].tolist() for i in range(len(off) - 1)] == \
        [f.tolist() for f in wf]


def test_sharded_2d_more_ranks_than_points():
    # 8 ranks over 5 and 9 points: some shards are empty, the result is still
    # the whole cloud's hull
    from paper_1201_2936_gb300 import build
    build.build()
    oracle.build()
    rng = np.random.default_rng(99)
    clouds = [tuple(rng.random((2, 5)).astype(np.float32)),
              tuple(rng.random((2, 9)).astype(np.float32))]
    hulls, st = _simulated(clouds, 8, cap=64)
    assert st == [0, 0]
    for h, (x, y) in zip(hulls, clouds):
        assert h.cpu().numpy().tolist() == oracle.hull2d(x, y).tolist()
