"""GPU parity of the segmented primitives (flagPermute, Algorithm 2; compact,
Algorithm 3) against the oracle's restatement, element by element (integer,
bit-exact), including Figure 1's worked example; and of the k-th element
selection built on them against the plain definition."""
import os

import numpy as np
import pytest
import torch

import oracle
from oracle import segmented as S

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def qh():
    from paper_1201_2936_gb300 import build
    build.build()
    import paper_1201_2936_gb300 as q
    return q


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(np.asarray(a, dtype=np.int32))).cuda()


def _golden():
    rows = {}
    with open(os.path.join(HERE, "golden", "fig1_flagpermute.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            name, *vals = line.split()
            rows[name] = np.array([int(x) for x in vals])
    return rows


def test_figure1(qh):
    g = _golden()
    p, s_new = qh.flag_permute(_t(g["f"]), _t(g["s"]), 3)
    assert p.cpu().numpy().tolist() == g["p"].tolist()
    assert s_new.cpu().numpy().tolist() == g["s_new"].tolist()


def _random_case(rng, n, k, pseg):
    f = rng.integers(0, k, n)
    s = (rng.random(n) < pseg).astype(np.int64)
    s[0] = 1
    return f, s


@pytest.mark.parametrize("n,k,pseg", [(1, 2, 0.5), (37, 2, 0.1), (4095, 3, 0.01), (4097, 3, 0.5),
                                      (20_011, 4, 0.001), (50_000, 7, 0.05), (65_537, 2, 0.0)])
def test_flag_permute_matches_oracle(qh, n, k, pseg):
    rng = np.random.default_rng(n + k)
    f, s = _random_case(rng, n, k, pseg)
    want_p, want_s, _ = S.flag_permute(f, s, k)
    p, s_new = qh.flag_permute(_t(f), _t(s), k)
    assert p.cpu().numpy().tolist() == want_p.tolist()
    assert s_new.cpu().numpy().tolist() == want_s.tolist()


@pytest.mark.parametrize("n,ptrue,pseg", [(1, 1.0, 0.5), (64, 0.5, 0.2), (4096, 0.3, 0.02),
                                          (30_001, 0.05, 0.01), (50_000, 0.0, 0.1),
                                          (65_537, 1.0, 0.001)])
def test_compact_matches_oracle(qh, n, ptrue, pseg):
    rng = np.random.default_rng(n)
    b = (rng.random(n) < ptrue).astype(np.int64)
    s = (rng.random(n) < pseg).astype(np.int64)
    s[0] = 1
    want_p, _, want_n, want_s = S.compact(b, s)
    p, s_new, nn = qh.compact(_t(b), _t(s))
    assert nn == want_n
    assert p.cpu().numpy().tolist() == want_p.tolist()
    assert s_new.cpu().numpy().tolist() == want_s.tolist()


def test_bad_states_are_rejected(qh):
    with pytest.raises(qh.QHError) as ei:
        qh.flag_permute(_t([0, 1, 3]), _t([1, 0, 0]), 3)
    assert ei.value.status == 1


def _sel_case(rng, nseg, lo, hi, kind):
    sizes = rng.integers(lo, hi + 1, nseg)
    off = np.zeros(nseg + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    n = int(off[-1])
    if kind == "uniform":
        v = rng.random(n).astype(np.float32)
    elif kind == "ties":
        v = rng.integers(0, 5, n).astype(np.float32)
    elif kind == "sorted":
        v = np.concatenate([np.sort(rng.random(s)) for s in sizes]).astype(np.float32)
    else:
        v = rng.standard_normal(n).astype(np.float32)
        v[rng.integers(0, n, 7)] = np.float32(-0.0)
        v[rng.integers(0, n, 7)] = np.float32(0.0)
    k = np.array([rng.integers(0, s) for s in sizes], np.int64)
    return v, off, k


@pytest.mark.parametrize("kind", ["uniform", "ties", "sorted", "signed-zeros"])
def test_select_matches_definition(qh, kind):
    rng = np.random.default_rng(len(kind))
    v, off, k = _sel_case(rng, 300, 1, 3000, kind)
    want = oracle.select(v, off, k)
    got = qh.select(torch.from_numpy(v).cuda(), torch.from_numpy(off).cuda(),
                    torch.from_numpy(k).cuda())
    assert got.cpu().numpy().tolist() == want.tolist()


def test_select_medians_large_batch(qh):
    # the selection workload: medians of 4096 segments of 4096 values
    rng = np.random.default_rng(9)
    v = rng.standard_normal(4096 * 4096).astype(np.float32)
    off = np.arange(4097, dtype=np.int64) * 4096
    k = np.full(4096, 2047, np.int64)
    want = oracle.select(v, off, k)
    got = qh.select(torch.from_numpy(v).cuda(), torch.from_numpy(off).cuda(),
                    torch.from_numpy(k).cuda())
    assert got.cpu().numpy().tolist() == want.tolist()


def test_select_rejects_bad_ranks(qh):
    v = torch.zeros(10, device="cuda")
    off = torch.tensor([0, 4, 10], dtype=torch.int64, device="cuda")
    with pytest.raises(qh.QHError):
        qh.select(v, off, torch.tensor([4, 0], dtype=torch.int64, device="cuda"))


@pytest.mark.parametrize("sizes", [[300_000, 9000, 4097, 1, 4096, 250_001],
                                   [1_000_000], [5000] * 40 + [3] * 17])
def test_select_long_segments_device_rounds(qh, sizes):
    # segments above 4096 elements go through the grid-wide rounds (the kept
    # parts move to shared-memory tasks once they are short): equal to the
    # definition, and to the host loop result for result and round for round
    rng = np.random.default_rng(sum(sizes) % 1000)
    n = sum(sizes)
    v = rng.standard_normal(n).astype(np.float32)
    v[rng.integers(0, n, n // 10)] = np.float32(0.5)  # ties, ordered by index
    off = np.zeros(len(sizes) + 1, np.int64)
    off[1:] = np.cumsum(sizes)
    k = np.array([rng.integers(0, s) for s in sizes], np.int64)
    want = oracle.select(v, off, k)
    V, O, K = (torch.from_numpy(a).cuda() for a in (v, off, k))
    got, it_d = qh.select(V, O, K, return_iters=True)
    host, it_h = qh.select(V, O, K, return_iters=True, loop="host")
    assert got.cpu().numpy().tolist() == want.tolist()
    assert host.cpu().numpy().tolist() == want.tolist()
    assert it_d == it_h


def test_select_device_and_host_rounds_agree_on_medians(qh):
    rng = np.random.default_rng(19)
    v = rng.standard_normal(512 * 4096).astype(np.float32)
    off = np.arange(513, dtype=np.int64) * 4096
    k = np.full(512, 2047, np.int64)
    V, O, K = (torch.from_numpy(a).cuda() for a in (v, off, k))
    got, it_d = qh.select(V, O, K, return_iters=True)
    host, it_h = qh.select(V, O, K, return_iters=True, loop="host")
    assert got.cpu().tolist() == host.cpu().tolist() == oracle.select(v, off, k).tolist()
    assert it_d == it_h


def test_select_edge_cases_device_loop(qh):
    # NaNs (ordered at the ends by their bits), every segment of one element,
    # and one long segment (global rounds) at its first and last rank
    rng = np.random.default_rng(23)
    v = rng.standard_normal(20_000).astype(np.float32)
    v[rng.integers(0, 20_000, 50)] = np.float32(np.nan)
    v[rng.integers(0, 20_000, 50)] = -np.float32(np.nan)
    off = np.array([0, 9_000, 9_001, 20_000], np.int64)
    for k in ([0, 0, 0], [8_999, 0, 10_998], [4_500, 0, 5_000]):
        k = np.array(k, np.int64)
        want = oracle.select(v, off, k)
        got = qh.select(torch.from_numpy(v).cuda(), torch.from_numpy(off).cuda(),
                        torch.from_numpy(k).cuda())
        assert got.cpu().numpy().tolist() == want.tolist(), k
    n = 3000
    v1 = rng.standard_normal(n).astype(np.float32)
    off1 = np.arange(n + 1, dtype=np.int64)
    k1 = np.zeros(n, np.int64)
    got = qh.select(torch.from_numpy(v1).cuda(), torch.from_numpy(off1).cuda(),
                    torch.from_numpy(k1).cuda())
    assert got.cpu().numpy().tolist() == list(range(n))
    big = rng.standard_normal(150_000).astype(np.float32)
    offb = np.array([0, 150_000], np.int64)
    for kk in (0, 149_999, 77_777):
        kb = np.array([kk], np.int64)
        got = qh.select(torch.from_numpy(big).cuda(), torch.from_numpy(offb).cuda(),
                        torch.from_numpy(kb).cuda())
        assert got.cpu().numpy().tolist() == oracle.select(big, offb, kb).tolist(), kk
