"""Pins for the restated flagPermute (Algorithm 2) and compact (Algorithm 3).

Figure 1 fixes every intermediate row of a 3-state flagPermute.  The test
shows that the printed mask/scan/backscan rows follow the listing literally,
that the printed permutation and new heads follow only when the backward
scan is read as the per-segment count, and checks the compact behaviour the
Figure 2 caption and Section 4.2 describe.
"""
import os

import numpy as np

import oracle
from oracle import segmented as sg

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    rows = {}
    with open(os.path.join(HERE, "golden", "fig1_flagpermute.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            k, *v = line.split()
            rows[k] = np.array([int(t) for t in v])
    return rows


def test_figure1_rows_literal_listing():
    g = _golden()
    p, s_new, rows = sg.flag_permute(g["f"], g["s"], 3, literal_backscan=True)
    assert rows["s_t"].tolist() == g["s_t"].tolist()
    assert rows["s_h"].tolist() == g["s_h"].tolist()
    for i in range(3):
        assert rows["mask"][i].tolist() == g[f"mask{i}"].tolist()
        assert rows["scan"][i].tolist() == g[f"scan{i}"].tolist()
    for i in range(2):
        assert rows["backscan"][i].tolist() == g[f"backscan{i}"].tolist()
    # the literal backward max does not give the printed permutation
    assert p.tolist() != g["p"].tolist()
    assert len(set(p.tolist())) < len(p)


def test_figure1_permutation_and_heads():
    g = _golden()
    p, s_new, _ = sg.flag_permute(g["f"], g["s"], 3)
    assert p.tolist() == g["p"].tolist()
    assert s_new.tolist() == g["s_new"].tolist()


def test_flag_permute_random_properties():
    rng = np.random.default_rng(0)
    for _ in range(200):
        n = int(rng.integers(1, 40))
        k = int(rng.integers(1, 5))
        f = rng.integers(0, k, n)
        s = (rng.random(n) < 0.2).astype(int)
        s[0] = 1
        p, s_new, _ = sg.flag_permute(f, s, k)
        assert sorted(p.tolist()) == list(range(n))          # a permutation
        seg = np.cumsum(s) - 1
        fp = sg.apply_permutation(f, p)
        segp = sg.apply_permutation(seg, p)
        assert np.all(np.diff(segp) >= 0)                     # segments stay in place
        for j in np.unique(seg):
            idx = np.where(segp == j)[0]
            assert np.all(np.diff(fp[idx]) >= 0)              # grouped by state
        # stable within a (segment, state) group
        for j in range(n):
            for i in range(j):
                if seg[i] == seg[j] and f[i] == f[j]:
                    assert p[i] < p[j]
        # new heads: exactly where (segment, state) changes in the output
        want = np.zeros(n, int)
        want[0] = 1
        for i in range(1, n):
            if segp[i] != segp[i - 1] or fp[i] != fp[i - 1]:
                want[i] = 1
        assert s_new.tolist() == want.tolist()


def test_compact_head_moves_and_segment_dies():
    # segment heads at 0, 3, 5; in the second segment both elements are false,
    # so its head is lost (Figure 2 caption); in the first the head moves to
    # the first true element (Section 4.2, case 1)
    b = np.array([0, 1, 1, 0, 0, 1, 0, 1])
    s = np.array([1, 0, 0, 1, 0, 1, 0, 0])
    p, sp, n_new, s_new = sg.compact(b, s)
    assert p.tolist() == [0, 0, 1, 2, 2, 2, 3, 3]
    assert n_new == 4
    assert sp[0] == 0 and sp[3] == sg.INF and sp[5] == 2
    assert s_new.tolist() == [1, 0, 1, 0]


def test_compact_random_properties():
    rng = np.random.default_rng(1)
    for _ in range(200):
        n = int(rng.integers(1, 40))
        b = (rng.random(n) < 0.5).astype(int)
        s = (rng.random(n) < 0.25).astype(int)
        s[0] = 1
        p, sp, n_new, s_new = sg.compact(b, s)
        keep = np.where(b == 1)[0]
        assert n_new == len(keep)
        assert p[keep].tolist() == list(range(n_new))
        seg = np.cumsum(s) - 1
        want = np.zeros(n_new, int)
        for i, src in enumerate(keep):
            if i == 0 or seg[keep[i - 1]] != seg[src]:
                want[i] = 1
        assert s_new.tolist() == want.tolist()


def test_select_oracle_against_sorting_and_ties():
    # the selection oracle: for distinct values it is the k-th entry of the
    # sorted segment; ties go to the lower index; -0.0 sorts before +0.0
    rng = np.random.default_rng(4)
    v = rng.permutation(200).astype(np.float32)
    off = np.array([0, 50, 51, 200])
    k = np.array([10, 0, 148])
    got = oracle.select(v, off, k)
    for c in range(3):
        seg = v[off[c]:off[c + 1]]
        assert v[got[c]] == np.sort(seg)[k[c]]
    t = np.array([3, 1, 3, 1, 3], np.float32)
    assert oracle.select(t, [0, 5], [0]).tolist() == [1]
    assert oracle.select(t, [0, 5], [1]).tolist() == [3]
    assert oracle.select(t, [0, 5], [2]).tolist() == [0]
    assert oracle.select(t, [0, 5], [4]).tolist() == [4]
    z = np.array([0.0, -0.0, -1.0], np.float32)
    assert oracle.select(z, [0, 3], [1]).tolist() == [1]
