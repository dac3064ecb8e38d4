"""GPU parity of the batched 2D hull (qh_hull2d_batched): every cloud's
hull equals the oracle's on a mixed batch of edge cases, on the
differentiable-hull workload (1024 clouds of 4096 points in the disk) and
after a CUDA-graph replay."""
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


def _batch(clouds):
    off = np.zeros(len(clouds) + 1, np.int64)
    off[1:] = np.cumsum([len(c[0]) for c in clouds])
    x = np.ascontiguousarray(np.concatenate([c[0] for c in clouds]).astype(np.float32))
    y = np.ascontiguousarray(np.concatenate([c[1] for c in clouds]).astype(np.float32))
    return x, y, off


def _mixed(seed):
    rng = np.random.default_rng(seed)
    clouds = []
    for k in range(30):
        n = int(np.exp(rng.uniform(np.log(3), np.log(20000))))
        kind = k % 5
        if kind == 0:
            r, t = np.sqrt(rng.random(n)), 2 * np.pi * rng.random(n)
            clouds.append((r * np.cos(t), r * np.sin(t)))
        elif kind == 1:
            clouds.append((rng.random(n), rng.random(n)))
        elif kind == 2:
            t = 2 * np.pi * rng.random(n)
            clouds.append((np.cos(t), np.sin(t)))            # nearly all on the hull
        elif kind == 3:
            clouds.append(tuple(rng.integers(-4, 5, (2, n))))  # lattice: collinear ties
        else:
            base = rng.random((2, 7))
            clouds.append(tuple(base[:, rng.integers(0, 7, n)]))  # duplicates
    t = rng.random(50)
    extras = [(np.zeros(0), np.zeros(0)), (np.array([0.3]), np.array([0.7])),
              (np.full(9, 0.25), np.full(9, -1.0)), (t, 2 * t + 1),
              (np.array([0.0, np.nan, 1.0]), np.array([0.0, 0.0, 1.0])),
              (np.array([1.0, 0.0]), np.array([1.0, 0.0]))]
    for e in extras:
        clouds.insert(int(rng.integers(0, len(clouds) + 1)), e)
    return _batch(clouds)


def _want(x, y, off):
    out = []
    for c in range(len(off) - 1):
        a, b = int(off[c]), int(off[c + 1])
        try:
            out.append((0, (oracle.hull2d(x[a:b], y[a:b]) + a).tolist()))
        except oracle.OracleError as e:
            out.append((e.code, []))
    return out


def _got(off, res):
    out, cnt, st = (t.cpu().numpy() for t in res)
    return [(int(st[c]), out[off[c]:off[c] + cnt[c]].tolist()) for c in range(len(off) - 1)]


def test_mixed_batch_matches_oracle(qh):
    x, y, off = _mixed(3)
    want = _want(x, y, off)
    P = torch.from_numpy(np.stack([x, y])).cuda()
    O = torch.from_numpy(off).cuda()
    for pred in ("f32", "f64"):
        got = _got(off, qh.hull2d_batched(P, cloud_off=O, pred=pred))
        for c, (g, e) in enumerate(zip(got, want)):
            assert g == e, (pred, c)


def test_interleaved_and_graph_replay(qh):
    x, y, off = w.batched_disk_2d(200, 1000, 17)
    want = _want(x, y, off)
    P = torch.from_numpy(np.stack([x, y], 1)).cuda()  # [n, 2]
    b = qh.Hull2DBatch(P, cloud_off=torch.from_numpy(off).cuda())
    b.capture()
    for _ in range(2):
        b.out.fill_(-1)
        b.replay()
        torch.cuda.synchronize()
        assert _got(off, b.outputs()) == want


def test_bad_offsets(qh):
    x, y, off = w.batched_disk_2d(4, 100, 1)
    bad = off.copy()
    bad[-1] += 1
    P = torch.from_numpy(np.stack([x, y])).cuda()
    b = qh.Hull2DBatch(P, cloud_off=torch.from_numpy(bad).cuda())
    b.enqueue()
    with pytest.raises(qh.QHError) as ei:
        b.outputs()
    assert ei.value.status == 1


def test_full_batch_1024_disks(qh):
    # the 2D differentiable-hull workload: 1024 clouds x 4096 points in the disk
    x, y, off = w.batched_disk_2d(1024, 4096, w.SEED_BASE + 4)
    want = _want(x, y, off)
    P = torch.from_numpy(np.stack([x, y])).cuda()
    got = _got(off, qh.hull2d_batched(P, cloud_off=torch.from_numpy(off).cuda()))
    assert got == want
