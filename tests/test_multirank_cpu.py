"""The multi-rank hull (paper_1201_2936_gb300.shard) on CPU ranks with gloo,
world sizes 2 to 4: the hull of the gathered shard hulls equals the oracle's
hull of the whole cloud (2D: the vertex list in order; 3D: the vertices and
the canonical face list), including duplicates across shards, shards with
no points and 3D shards that do not span space (fewer than four points, or
coplanar), whose points are all candidates."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

import oracle
from paper_1201_2936_gb300 import shard
from paper_1201_2936_gb300 import workloads as w


def test_shard_ranges_cover_exactly():
    for n in (0, 1, 5, 100, 101):
        for world in (1, 2, 3, 7):
            rs = [shard.shard_range(n, r, world) for r in range(world)]
            assert rs[0][0] == 0 and rs[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(rs, rs[1:]))
            assert max(h - l for l, h in rs) - min(h - l for l, h in rs) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _oracle3d_or_none(c):
    # the shard-hull protocol: None for points that do not span 3D
    try:
        return oracle.hull3d(c[0], c[1], c[2])
    except oracle.OracleError as e:
        if e.code == 3:
            return None
        raise


def _cloud3d(case):
    if case == "tiny":  # shards of 2 or 3 points: none spans 3D
        r = np.random.default_rng(79)
        return tuple(r.uniform(-1, 1, (3, 9)).astype(np.float32))
    if case == "coplanar":  # the middle shard on one plane inside the ball
        x, y, z = (c[:3000] for c in w.uniform_ball(3000, 80))
        z = z.copy()
        z[1000:2000] = np.float32(0.125)
        return x, y, z
    x, y, z = w.uniform_ball(6000, 78)
    # a duplicated hull vertex in a later shard, and a cube corner set with
    # coplanar (quadrilateral) faces
    x = np.concatenate([x, x[:30], np.float32([2, 2, 2, 2])]).astype(np.float32)
    y = np.concatenate([y, y[:30], np.float32([2, 2, -2, -2])]).astype(np.float32)
    z = np.concatenate([z, z[:30], np.float32([2, -2, 2, -2])]).astype(np.float32)
    return x, y, z


def _worker(rank, world, port, dim, q, case="ball"):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        oracle.build()
        if dim == 2:
            x, y = w.uniform_disk(20000, 77)
            # duplicates of a hull vertex in a later shard, and a far point
            x = np.concatenate([x, x[:50], np.float32([3.0])]).astype(np.float32)
            y = np.concatenate([y, y[:50], np.float32([0.25])]).astype(np.float32)
            final, _ = shard.sharded_hull_numpy([x, y], lambda c: oracle.hull2d(c[0], c[1]))
            want = oracle.hull2d(x, y)
        else:
            x, y, z = _cloud3d(case)
            fv, ff = shard.sharded_hull3d_numpy([x, y, z], _oracle3d_or_none)
            wv, wf = oracle.hull3d(x, y, z)
            final = (fv.tolist(), [f.tolist() for f in ff])
            want = (wv.tolist(), [f.tolist() for f in wf])
            q.put((rank, final, want))
            return
        q.put((rank, final.tolist(), want.tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,dim,case", [(2, 2, "ball"), (3, 2, "ball"), (2, 3, "ball"),
                                            (3, 3, "ball"), (3, 3, "tiny"), (4, 3, "tiny"),
                                            (3, 3, "coplanar")])
def test_sharded_hull_equals_whole_hull(world, dim, case):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, dim, q, case))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, final, want in res:
        assert final == want, rank


def test_one_rank_degenerate_cloud_raises_and_gpu_hull_maps_the_status(monkeypatch):
    from paper_1201_2936_gb300 import build
    build.build()
    oracle.build()
    import paper_1201_2936_gb300 as qh
    # the whole cloud on one plane: the final hull is degenerate too
    x, y, z = (c[:500] for c in w.uniform_ball(500, 81))
    z = np.zeros_like(z)
    with pytest.raises(qh.QHError) as e:
        shard.sharded_hull3d_numpy([x, y, z], _oracle3d_or_none)
    assert e.value.status == shard.QH_ERR_DEGENERATE
    # the library's hull functions: QH_ERR_DEGENERATE -> None, others raise
    pts = [torch.zeros(4), torch.zeros(4), torch.zeros(4)]

    def raising(status):
        def f(*a, **k):
            raise qh.QHError(status, "qh_hull3d")
        return f

    monkeypatch.setattr(qh, "hull3d", raising(3))
    assert shard._gpu_hull(pts) is None and shard._gpu_hull3d_faces(pts) is None
    monkeypatch.setattr(qh, "hull3d", raising(8))
    for fn in (shard._gpu_hull, shard._gpu_hull3d_faces):
        with pytest.raises(qh.QHError):
            fn(pts)
