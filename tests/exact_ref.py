"""Exact rational references used to pin the oracle (Python Fractions).

These restate only textbook definitions (determinants, brute-force hull
tests, Andrew's monotone chain); none of the hull code under test is used.
"""
from __future__ import annotations

from fractions import Fraction
from itertools import combinations

import numpy as np


def F(v) -> Fraction:
    return Fraction(float(v))


def orient2d(a, b, c) -> int:
    ax, ay, bx, by, cx, cy = (F(v) for v in (a[0], a[1], b[0], b[1], c[0], c[1]))
    d = (ax - cx) * (by - cy) - (ay - cy) * (bx - cx)
    return (d > 0) - (d < 0)


def det3(u, v, w) -> Fraction:
    return (u[0] * (v[1] * w[2] - v[2] * w[1]) - u[1] * (v[0] * w[2] - v[2] * w[0])
            + u[2] * (v[0] * w[1] - v[1] * w[0]))


def orient3d(a, b, c, p) -> int:
    A, B, C, P = ([F(t) for t in q] for q in (a, b, c, p))
    u = [B[i] - A[i] for i in range(3)]
    v = [C[i] - A[i] for i in range(3)]
    w = [P[i] - A[i] for i in range(3)]
    d = det3(u, v, w)
    return (d > 0) - (d < 0)


def unique_lowest(points):
    """Map each location to its lowest index; points is a list of tuples."""
    best = {}
    for i, p in enumerate(points):
        key = tuple(float(v) + 0.0 for v in p)
        if key not in best:
            best[key] = i
    return best


def brute_hull2d(x, y):
    """CCW extreme points from the lexicographic minimum by the O(n^3) edge
    test: (i, j) is a hull edge when every point is left of or on i->j and
    every point on the line lies in the closed segment [i, j]."""
    pts = list(zip(np.asarray(x, np.float64).tolist(), np.asarray(y, np.float64).tolist()))
    if not pts:
        return []
    loc = unique_lowest(pts)
    ids = sorted(loc.values())
    if len(ids) == 1:
        return ids
    P = {i: (F(pts[i][0]), F(pts[i][1])) for i in ids}
    succ = {}
    for i in ids:
        for j in ids:
            if i == j:
                continue
            ok = True
            for k in ids:
                s = orient2d(P[i], P[j], P[k])
                if s < 0:
                    ok = False
                    break
                if s == 0:
                    # k must lie in the closed segment [i, j]
                    lo = (min(P[i][0], P[j][0]), min(P[i][1], P[j][1]))
                    hi = (max(P[i][0], P[j][0]), max(P[i][1], P[j][1]))
                    if not (lo[0] <= P[k][0] <= hi[0] and lo[1] <= P[k][1] <= hi[1]):
                        ok = False
                        break
            if ok:
                succ.setdefault(i, []).append(j)
    start = min(ids, key=lambda i: (P[i][0], P[i][1]))
    out = [start]
    cur = start
    while True:
        nxt = succ[cur][0]
        if nxt == start:
            break
        out.append(nxt)
        cur = nxt
        assert len(out) <= len(ids)
    return out


def monotone_chain2d(x, y):
    """Andrew's monotone chain with exact orientation, duplicates removed
    first (lowest index kept); CCW from the lexicographic minimum."""
    pts = list(zip(np.asarray(x, np.float64).tolist(), np.asarray(y, np.float64).tolist()))
    if not pts:
        return []
    loc = unique_lowest(pts)
    order = sorted(loc.items(), key=lambda kv: kv[0])
    ids = [i for _, i in order]
    P = {i: (F(pts[i][0]), F(pts[i][1])) for i in ids}
    if len(ids) <= 2:
        return ids

    def half(seq):
        h = []
        for i in seq:
            while len(h) >= 2 and orient2d(P[h[-2]], P[h[-1]], P[i]) <= 0:
                h.pop()
            h.append(i)
        return h

    lower = half(ids)
    upper = half(ids[::-1])
    hull = lower[:-1] + upper[:-1]
    if len(hull) == 2 and hull[0] == hull[1]:
        return hull[:1]
    return hull


def _hull2d_of_projected(ids, P3, drop):
    keep = [k for k in range(3) if k != drop]
    proj = {i: (P3[i][keep[0]], P3[i][keep[1]]) for i in ids}
    order = sorted(ids, key=lambda i: proj[i])
    if len(order) <= 2:
        return order

    def half(seq):
        h = []
        for i in seq:
            while len(h) >= 2 and orient2d(proj[h[-2]], proj[h[-1]], proj[i]) <= 0:
                h.pop()
            h.append(i)
        return h

    lo = half(order)
    up = half(order[::-1])
    return lo[:-1] + up[:-1]


def brute_hull3d(x, y, z):
    """Canonical face list by brute force: every supporting plane through
    three non-collinear points, its coplanar points' 2D hull as the face,
    oriented CCW from outside, rotated to the smallest index, faces sorted.
    Returns (sorted vertex list, list of face tuples) or None if the points
    do not span 3D."""
    pts = list(zip(*(np.asarray(c, np.float64).tolist() for c in (x, y, z))))
    loc = unique_lowest(pts)
    ids = sorted(loc.values())
    P = {i: tuple(F(v) for v in pts[i]) for i in ids}
    faces = {}
    spans = False
    for i, j, k in combinations(ids, 3):
        u = [P[j][t] - P[i][t] for t in range(3)]
        v = [P[k][t] - P[i][t] for t in range(3)]
        nrm = (u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0])
        if nrm == (0, 0, 0):
            continue
        side = []
        for m in ids:
            w = [P[m][t] - P[i][t] for t in range(3)]
            d = nrm[0] * w[0] + nrm[1] * w[1] + nrm[2] * w[2]
            side.append((d > 0) - (d < 0))
        if any(s != 0 for s in side):
            spans = True
        if all(s <= 0 for s in side):
            out_n = nrm
        elif all(s >= 0 for s in side):
            out_n = tuple(-c for c in nrm)
        else:
            continue
        cop = frozenset(m for m, s in zip(ids, side) if s == 0)
        faces[cop] = out_n
    if not spans:
        return None
    result = []
    for cop, out_n in faces.items():
        drop = max(range(3), key=lambda t: abs(out_n[t]))
        poly = _hull2d_of_projected(sorted(cop), P, drop)
        # orient CCW seen from outside
        a, b, c = P[poly[0]], P[poly[1]], P[poly[2]]
        u = [b[t] - a[t] for t in range(3)]
        v = [c[t] - b[t] for t in range(3)]
        cr = (u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0])
        if sum(cr[t] * out_n[t] for t in range(3)) < 0:
            poly = poly[::-1]
        r = poly.index(min(poly))
        result.append(tuple(poly[r:] + poly[:r]))
    result.sort()
    verts = sorted({v for f in result for v in f})
    return verts, result


# ---------------------------------------------------------------- 4D

def det4(rows) -> Fraction:
    """Determinant of a 4x4 matrix of Fractions by cofactor expansion."""
    def det3r(m):
        return det3(m[0], m[1], m[2])
    tot = Fraction(0)
    for j in range(4):
        minor = [[rows[i][k] for k in range(4) if k != j] for i in range(1, 4)]
        term = rows[0][j] * det3r(minor)
        tot += term if j % 2 == 0 else -term
    return tot


def orient4(a, b, c, d, p) -> int:
    """Sign of det[b-a; c-a; d-a; p-a] in exact rationals."""
    A, B, C, D, P = ([F(t) for t in q] for q in (a, b, c, d, p))
    d4 = det4([[B[i] - A[i] for i in range(4)], [C[i] - A[i] for i in range(4)],
               [D[i] - A[i] for i in range(4)], [P[i] - A[i] for i in range(4)]])
    return (d4 > 0) - (d4 < 0)


def _normal4(A, B, C, D):
    """A normal of the hyperplane through four points (Fractions): the
    generalised cross product of b-a, c-a, d-a (zero vector when they are
    affinely dependent)."""
    u = [B[i] - A[i] for i in range(4)]
    v = [C[i] - A[i] for i in range(4)]
    w = [D[i] - A[i] for i in range(4)]
    n = []
    for j in range(4):
        cols = [k for k in range(4) if k != j]
        m = det3([u[k] for k in cols], [v[k] for k in cols], [w[k] for k in cols])
        n.append(m if j % 2 == 0 else -m)
    return n


def _rank(vecs) -> int:
    """Rank of a list of Fraction vectors (Gaussian elimination)."""
    rows = [list(v) for v in vecs]
    rank, col = 0, 0
    ncol = len(rows[0]) if rows else 0
    while rank < len(rows) and col < ncol:
        piv = next((r for r in range(rank, len(rows)) if rows[r][col] != 0), None)
        if piv is None:
            col += 1
            continue
        rows[rank], rows[piv] = rows[piv], rows[rank]
        for r in range(len(rows)):
            if r != rank and rows[r][col] != 0:
                f = rows[r][col] / rows[rank][col]
                rows[r] = [x - f * y for x, y in zip(rows[r], rows[rank])]
        rank += 1
        col += 1
    return rank


def brute_hull4d(x, y, z, w):
    """The 4D hull by definition, in exact rationals: every hyperplane through
    four affinely independent input locations with all points on one side is
    a supporting hyperplane, the points on it form a facet; a point is a
    vertex when the normals of the facets through it span R^4.  Returns
    (sorted vertex indices, sorted list of facet tuples of the vertices on
    each facet), or None when the points do not span R^4."""
    pts = list(zip(*(np.asarray(c, np.float64).tolist() for c in (x, y, z, w))))
    loc = unique_lowest(pts)
    ids = sorted(loc.values())
    P = {i: [F(t) for t in pts[i]] for i in ids}
    facets = {}
    for quad in combinations(ids, 4):
        A, B, C, D = (P[i] for i in quad)
        nrm = _normal4(A, B, C, D)
        if all(t == 0 for t in nrm):
            continue
        s = {i: sum(nrm[k] * (P[i][k] - A[k]) for k in range(4)) for i in ids}
        if all(v >= 0 for v in s.values()) or all(v <= 0 for v in s.values()):
            on = frozenset(i for i in ids if s[i] == 0)
            if len(on) == len(ids):
                return None  # every point on one hyperplane
            facets[on] = nrm
    if not facets:
        return None
    verts = []
    for i in ids:
        normals = [nrm for on, nrm in facets.items() if i in on]
        if normals and _rank(normals) == 4:
            verts.append(i)
    vset = set(verts)
    out = sorted(tuple(sorted(i for i in on if i in vset)) for on in facets)
    return verts, out
