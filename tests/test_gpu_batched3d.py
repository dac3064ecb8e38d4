"""GPU parity of the batched 3D hull (qh_hull3d_batched): every cloud's
status, vertex list and canonical face list equal the oracle's loop over the
clouds; identical outputs for every launch shape, for a CUDA-graph replay and
after autotuning; the full 4096-cloud batch of anisotropic Gaussian clouds."""
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


def _mixed_batch(seed):
    """Gaussian clouds of log-uniform sizes plus the edge cases: an empty
    cloud, 1 and 3 points, a coplanar cloud, a cloud with a NaN, a lattice
    cloud (coplanar faces), points on a sphere, duplicates."""
    x, y, z, off = w.batched_clouds_3d(40, seed, nmin=16, nmax=4096)
    clouds = [tuple(c[off[i]:off[i + 1]] for c in (x, y, z)) for i in range(40)]
    rng = np.random.default_rng(seed)
    extra = [np.zeros((3, 0)), rng.random((3, 1)), rng.random((3, 3))]
    flat = rng.random((3, 50))
    flat[1] = 0.25
    extra.append(flat)
    bad = rng.random((3, 30))
    bad[0, 7] = np.nan
    extra.append(bad)
    extra.append(rng.integers(-2, 3, (3, 300)))
    g = rng.standard_normal((3, 2000))
    extra.append(g / np.linalg.norm(g, axis=0))
    base = rng.random((3, 6))
    extra.append(base[:, rng.integers(0, 6, 100)])
    for e in extra:
        clouds.insert(int(rng.integers(0, len(clouds) + 1)),
                      tuple(np.ascontiguousarray(c, np.float32) for c in e))
    off = np.zeros(len(clouds) + 1, np.int64)
    off[1:] = np.cumsum([len(c[0]) for c in clouds])
    x, y, z = (np.ascontiguousarray(np.concatenate([c[i] for c in clouds])) for i in range(3))
    return x, y, z, off


def _split(outs):
    verts, cvo, foff, fidx, cfo, cst = (t.cpu().numpy() for t in outs)
    res = []
    for c in range(len(cst)):
        v = verts[cvo[c]:cvo[c + 1]]
        faces = [fidx[foff[i]:foff[i + 1]].tolist() for i in range(cfo[c], cfo[c + 1])]
        res.append((int(cst[c]), v.tolist(), faces))
    return res


def _want(x, y, z, off):
    return [(st, v.tolist(), [f.tolist() for f in fs]) for st, v, fs in
            oracle.hull3d_batched(x, y, z, off)]


def _dev(x, y, z, off):
    P = torch.from_numpy(np.stack([x, y, z])).cuda()
    return P, torch.from_numpy(off).cuda()


def test_mixed_batch_matches_oracle(qh):
    x, y, z, off = _mixed_batch(41)
    want = _want(x, y, z, off)
    P, O = _dev(x, y, z, off)
    for pred in ("f32", "f64"):
        got = _split(qh.hull3d_batched(P, cloud_off=O, pred=pred))
        assert len(got) == len(want)
        for c, (g, e) in enumerate(zip(got, want)):
            assert g == e, (pred, c)


def test_launch_shapes_agree(qh):
    x, y, z, off = _mixed_batch(42)
    want = _want(x, y, z, off)
    P, O = _dev(x, y, z, off)
    for block in (128, 256, 512):
        for items in (2, 4, 8):
            o = qh.make_opts("f32", block=block, items=items)
            got = _split(qh.hull3d_batched(P, cloud_off=O, opts=o))
            assert got == want, (block, items)


def test_graph_replay_and_autotune(qh):
    x, y, z, off = w.batched_clouds_3d(300, 77, nmin=16, nmax=8192)
    want = _want(x, y, z, off)
    P, O = _dev(x, y, z, off)
    b = qh.Hull3DBatch(P, cloud_off=O)
    table = b.tune(reps=1)
    assert len(table) >= 9 and all(ms > 0 for *_, ms in table)
    assert _split(b.outputs()) == want
    b.capture()
    for _ in range(2):
        b.verts.fill_(-1)
        b.face_idx.fill_(-1)
        b.replay()
        torch.cuda.synchronize()
        assert _split(b.outputs()) == want


def test_bad_offsets_fail_cleanly(qh):
    x, y, z, off = w.batched_clouds_3d(8, 5, nmin=16, nmax=64)
    P = torch.from_numpy(np.stack([x, y, z])).cuda()
    bad = off.copy()
    bad[3], bad[4] = bad[4], bad[3]  # decreasing
    b = qh.Hull3DBatch(P, cloud_off=torch.from_numpy(bad).cuda())
    b.enqueue()
    with pytest.raises(qh.QHError) as ei:
        b.outputs()
    assert ei.value.status == 1


def test_full_batch_4096_clouds(qh):
    # the batched workload at full size (4096 anisotropic Gaussian clouds,
    # sizes log-uniform in [16, 65536]) in the configuration the benchmark
    # times: autotuned shape, replayed CUDA graph
    x, y, z, off = w.batched_clouds_3d(4096, w.SEED_BASE + 3)
    want = _want(x, y, z, off)
    P, O = _dev(x, y, z, off)
    b = qh.Hull3DBatch(P, cloud_off=O)
    b.tune(reps=1)
    b.capture()
    b.replay()
    torch.cuda.synchronize()
    got = _split(b.outputs())
    assert len(got) == 4096
    for c in range(4096):
        assert got[c] == want[c], c


@pytest.mark.parametrize("small", [16, 64, 512, 4096])
def test_small_cloud_route_matches_oracle(qh, small):
    # clouds of 4..small points hulled whole by one warp in the setup: the
    # mixed batch's degenerate, coplanar, non-finite, lattice, duplicated
    # and spherical clouds included
    x, y, z, off = _mixed_batch(43)
    want = _want(x, y, z, off)
    P, O = _dev(x, y, z, off)
    for pred in ("f32", "f64"):
        o = qh.make_opts(pred, small_cloud=small)
        got = _split(qh.hull3d_batched(P, cloud_off=O, opts=o))
        assert got == want, (pred, small)


def test_full_batch_small_cloud_route(qh):
    # the full batch with most clouds (4..4096 points) on the warp route
    x, y, z, off = w.batched_clouds_3d(4096, w.SEED_BASE + 3)
    want = _want(x, y, z, off)
    P, O = _dev(x, y, z, off)
    got = _split(qh.hull3d_batched(P, cloud_off=O, opts=qh.make_opts("f32", small_cloud=4096)))
    assert len(got) == 4096
    for c in range(4096):
        assert got[c] == want[c], c


def test_many_small_clouds_tuned(qh):
    # a batch of many small clouds (where the warp route wins): autotuned
    # threshold, outputs equal to the oracle's, and the same with the route off
    x, y, z, off = w.batched_clouds_3d(2048, 98, nmin=16, nmax=256)
    want = _want(x, y, z, off)
    P, O = _dev(x, y, z, off)
    b = qh.Hull3DBatch(P, cloud_off=O)
    table = b.tune(reps=1)
    assert {sc for *_, sc, ms in table} >= {0, 64, 256, 1024, 4096}
    assert _split(b.outputs()) == want
    got0 = _split(qh.hull3d_batched(P, cloud_off=O, opts=qh.make_opts("f32", small_cloud=0)))
    assert got0 == want


@pytest.mark.parametrize("small", [0, 256])
def test_facet_capacity_below_worst_case(qh, small):
    # qh_opts.max_facets below the worst case (6 n + 4 ncloud + 64): the
    # facet arrays shrink, the clouds' segment entries and the small-cloud
    # route's per-point scratch stay; every cloud still equals the oracle
    x, y, z, off = w.batched_clouds_3d(256, 44, nmin=16, nmax=8192)
    n, nc = len(x), len(off) - 1
    want = _want(x, y, z, off)
    P, O = _dev(x, y, z, off)
    o = qh.make_opts("f32", small_cloud=small, max_facets=3 * n + 4 * nc + 256)
    assert qh.workspace_bytes_3d_batched(n, nc, o) < qh.workspace_bytes_3d_batched(n, nc, None)
    got = _split(qh.hull3d_batched(P, cloud_off=O, opts=o))
    assert got == want
