"""Hull measures and their gradients in FP64 (test infrastructure: only
tests, the smoke check and the benchmark's CPU baseline use the oracle).

The paper computes hulls only; the measures make the hull a differentiable
layer.  Each function is the plain definition:
  2D (hull p_0..p_{h-1} counter-clockwise, indices cyclic)
    perimeter = sum_i |p_{i+1} - p_i|
    area      = 1/2 sum_i (x_i y_{i+1} - x_{i+1} y_i)          (shoelace)
  3D (faces counter-clockwise seen from outside, each split into the fan
      (f_0, f_k, f_{k+1}))
    area      = sum over fan triangles of |(b - a) x (c - a)| / 2
    volume    = sum over fan triangles of a . (b x c) / 6   (divergence theorem)
and the gradients are their partial derivatives with respect to the hull
vertices, written out term by term (every other point has gradient zero).
"""
from __future__ import annotations

import numpy as np


def _f64(a):
    return np.asarray(a, dtype=np.float64)


def measures2d(x, y, hull):
    """(perimeter, area) of the polygon hull (indices into x, y)."""
    x, y = _f64(x), _f64(y)
    h = len(hull)
    per = area = 0.0
    for i in range(h):
        a, b = hull[i], hull[(i + 1) % h]
        per += float(np.hypot(x[b] - x[a], y[b] - y[a]))
        area += 0.5 * float(x[a] * y[b] - x[b] * y[a])
    return per, area


def grad2d(x, y, hull, w_perim, w_area):
    """d(w_perim * perimeter + w_area * area) / d(x, y) for every point."""
    x, y = _f64(x), _f64(y)
    gx, gy = np.zeros(len(x)), np.zeros(len(y))
    h = len(hull)
    for i in range(h):
        v, prev, nxt = hull[i], hull[(i - 1) % h], hull[(i + 1) % h]
        # d|p_v - p_prev| / dp_v and d|p_next - p_v| / dp_v
        for o in (prev, nxt):
            dx, dy = x[v] - x[o], y[v] - y[o]
            ln = np.hypot(dx, dy)
            if ln > 0:
                gx[v] += w_perim * dx / ln
                gy[v] += w_perim * dy / ln
        # the shoelace terms holding p_v: x_prev y_v - x_v y_prev and x_v y_next - x_next y_v
        gx[v] += w_area * 0.5 * (y[nxt] - y[prev])
        gy[v] += w_area * 0.5 * (x[prev] - x[nxt])
    return gx, gy


def _fan(faces):
    for f in faces:
        for k in range(1, len(f) - 1):
            yield f[0], f[k], f[k + 1]


def measures3d(x, y, z, faces):
    """(surface area, volume) of the polyhedron with these faces."""
    P = np.stack([_f64(x), _f64(y), _f64(z)], axis=1)
    area = vol = 0.0
    for a, b, c in _fan(faces):
        pa, pb, pc = P[a], P[b], P[c]
        area += 0.5 * float(np.linalg.norm(np.cross(pb - pa, pc - pa)))
        vol += float(np.dot(pa, np.cross(pb, pc))) / 6.0
    return area, vol


def grad3d(x, y, z, faces, w_area, w_vol):
    """d(w_area * area + w_vol * volume) / d(x, y, z) for every point, as an
    [n, 3] array."""
    P = np.stack([_f64(x), _f64(y), _f64(z)], axis=1)
    g = np.zeros_like(P)
    for a, b, c in _fan(faces):
        pa, pb, pc = P[a], P[b], P[c]
        nrm = np.cross(pb - pa, pc - pa)
        ln = np.linalg.norm(nrm)
        if ln > 0:
            u = nrm / ln
            # |n| = u . n and dn = da x (b - c) + db x (c - a) + dc x (a - b)
            g[a] += w_area * 0.5 * np.cross(pb - pc, u)
            g[b] += w_area * 0.5 * np.cross(pc - pa, u)
            g[c] += w_area * 0.5 * np.cross(pa - pb, u)
        # a . (b x c) is linear in each vertex
        g[a] += w_vol * np.cross(pb, pc) / 6.0
        g[b] += w_vol * np.cross(pc, pa) / 6.0
        g[c] += w_vol * np.cross(pa, pb) / 6.0
    return g
