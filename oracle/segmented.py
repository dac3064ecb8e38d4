"""Restatement of the paper's segmented primitives: TEST INFRASTRUCTURE ONLY.

``flag_permute`` follows Algorithm 2 (k-state flagPermute, Section 4.1) and
``compact`` follows Algorithm 3 (Section 4.2), step by step in plain Python
loops over small arrays, with the readings needed where the printed listings
are garbled (each reading is stated at the step that uses it):

* Algorithm 2, the "backward inclusive max scan" of the exclusive scan is
  read as the per-segment total of the state (the count broadcast over the
  segment).  Figure 1's permutation and new heads are reproduced only under
  this reading; the literal backward max gives count - 1 when the segment's
  last element has the state, and no permutation.
* flagPermuteKernel's final line uses ``scan[i]`` after the loop; it is read
  as the scan of the element's own state ``f[id]``.
* addSegKernel sets a head at ``s_h + sum_{j<=i} count_j`` for each state
  boundary i < k-1 that lies inside the segment; old heads stay.  Empty state
  groups therefore add no head.
* Algorithm 3's ``segmented_scan(newSegment)`` is read as the backward
  inclusive segmented min of ``sp`` with identity +inf; a segment whose
  elements are all false loses its head (Figure 2 caption).
"""
from __future__ import annotations

import numpy as np

INF = np.iinfo(np.int64).max


def _segments(s):
    s = np.asarray(s)
    heads = [i for i in range(len(s)) if s[i] == 1 or i == 0]
    bounds = heads + [len(s)]
    return [(bounds[j], bounds[j + 1]) for j in range(len(heads))]


def segmented_scan_fwd_incl_sum(x, s):
    out = np.zeros(len(x), dtype=np.int64)
    acc = 0
    for i in range(len(x)):
        if i == 0 or s[i] == 1:
            acc = 0
        acc += int(x[i])
        out[i] = acc
    return out


def segmented_scan_fwd_excl_sum(x, s):
    out = np.zeros(len(x), dtype=np.int64)
    acc = 0
    for i in range(len(x)):
        if i == 0 or s[i] == 1:
            acc = 0
        out[i] = acc
        acc += int(x[i])
    return out


def segmented_scan_bwd_incl_max(x, s):
    """Literal Algorithm 2 step 13 (kept to show where the listing goes wrong)."""
    out = np.zeros(len(x), dtype=np.int64)
    for lo, hi in _segments(s):
        acc = None
        for i in range(hi - 1, lo - 1, -1):
            acc = int(x[i]) if acc is None else max(acc, int(x[i]))
            out[i] = acc
    return out


def segment_totals(x, s):
    """Per-segment total of x, broadcast over the segment (reading of
    Algorithm 2 step 13)."""
    out = np.zeros(len(x), dtype=np.int64)
    for lo, hi in _segments(s):
        out[lo:hi] = int(np.sum(np.asarray(x[lo:hi], dtype=np.int64)))
    return out


def flag_permute(f, s, k, literal_backscan: bool = False):
    """k-state flagPermute (Algorithm 2).

    Returns (p, s_new, rows) where p[id] is the destination of element id,
    s_new the new head flags and rows a dict of the intermediate arrays
    (s_t, s_h, mask[i], scan[i], backscan[i]) as in Figure 1.
    """
    f = np.asarray(f, dtype=np.int64)
    s = np.asarray(s, dtype=np.int64)
    n = len(f)
    # steps 1-5: s_t holds the index at heads, 0 elsewhere
    s_t = np.array([i if (s[i] == 1) else 0 for i in range(n)], dtype=np.int64)
    # step 7: forward inclusive segmented sum gives each element its head index
    s_h = segmented_scan_fwd_incl_sum(s_t, s)
    masks, scans, backs = [], [], []
    for i in range(k):
        m = (f == i).astype(np.int64)                    # steps 9, 14
        sc = segmented_scan_fwd_excl_sum(m, s)           # steps 11, 16
        masks.append(m)
        scans.append(sc)
        if literal_backscan:
            backs.append(segmented_scan_bwd_incl_max(sc, s))  # step 13 as printed
        else:
            backs.append(segment_totals(m, s))                # step 13, read as counts
    # flagPermuteKernel
    p = np.zeros(n, dtype=np.int64)
    for idx in range(n):
        loc = 0
        for i in range(int(f[idx])):
            loc += backs[i][idx]
        p[idx] = loc + s_h[idx] + scans[int(f[idx])][idx]
    # addSegKernel: old heads plus one head per state boundary inside the segment
    s_new = np.zeros(n, dtype=np.int64)
    for lo, hi in _segments(s):
        s_new[lo] = 1
        cum = 0
        for i in range(k - 1):
            cum += int(backs[i][lo])
            pos = lo + cum
            if pos < hi:
                s_new[pos] = 1
    rows = {"s_t": s_t, "s_h": s_h, "mask": masks, "scan": scans, "backscan": backs}
    return p, s_new, rows


def compact(b, s):
    """compact (Algorithm 3).

    Returns (p, sp, n_new, s_new): p is the exclusive scan of b (the
    destination of each true element), sp the backward inclusive segmented
    min of segmentMaskKernel's output (identity +inf), n_new the number of
    true elements and s_new the head flags of the compacted array (a segment
    with no true element disappears).
    """
    b = np.asarray(b, dtype=np.int64)
    s = np.asarray(s, dtype=np.int64)
    n = len(b)
    # step 2: forward exclusive (unsegmented) sum
    p = np.zeros(n, dtype=np.int64)
    acc = 0
    for i in range(n):
        p[i] = acc
        acc += int(b[i])
    # step 3: the number of true elements
    n_new = int(p[n - 1] + b[n - 1]) if n else 0
    # step 5: segmentMaskKernel
    out = np.array([p[i] if b[i] == 1 else INF for i in range(n)], dtype=np.int64)
    # step 7: backward inclusive segmented min
    sp = np.zeros(n, dtype=np.int64)
    for lo, hi in _segments(s):
        cur = INF
        for i in range(hi - 1, lo - 1, -1):
            cur = min(cur, int(out[i]))
            sp[i] = cur
    s_new = np.zeros(n_new, dtype=np.int64)
    for lo, hi in _segments(s):
        if sp[lo] != INF:
            s_new[sp[lo]] = 1
    return p, sp, n_new, s_new


def apply_permutation(values, p):
    out = np.empty_like(values)
    out[np.asarray(p)] = values
    return out
