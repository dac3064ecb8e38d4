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
