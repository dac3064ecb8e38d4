"""Oracle for segmented Quickhull: TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or runs anything here, and nothing
here uses the product path.

``qh_oracle.c`` is a plain sequential Quickhull in FP64 with exact predicates
(see its header); this module compiles it with gcc and wraps it with ctypes.
``segmented.py`` restates the paper's ``flagPermute`` (Algorithm 2) and
``compact`` (Algorithm 3) in numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_SRCS = [os.path.join(_HERE, "qh_oracle.c"), os.path.join(_HERE, "qh_oracle4.c")]
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID, ERR_NONFINITE, ERR_DEGENERATE, ERR_NOMEM = 0, 1, 2, 3, 4


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -ffp-contract=off so the FP64 error bounds hold)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or \
            any(os.path.getmtime(_SO) < os.path.getmtime(src) for src in _SRCS):
        tmp = _SO + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", tmp] + _SRCS + ["-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            fp = ctypes.c_void_p
            lib.oracle_hull2d.argtypes = [fp, fp, ctypes.c_int64, fp, i64p, i64p]
            lib.oracle_hull2d.restype = ctypes.c_int
            lib.oracle_hull3d.argtypes = [fp, fp, fp, ctypes.c_int64, fp, i64p, fp, fp, i64p, i64p]
            lib.oracle_hull3d.restype = ctypes.c_int
            lib.oracle_hull4d.argtypes = [fp, fp, fp, fp, ctypes.c_int64, fp, i64p, fp,
                                          ctypes.c_int64, fp, ctypes.c_int64, i64p, i64p]
            lib.oracle_hull4d.restype = ctypes.c_int
            for name, k in (("oracle_orient2d", 3), ("oracle_cmp_dist2", 4),
                            ("oracle_orient3d", 4), ("oracle_cmp_dist3", 5),
                            ("oracle_orient4", 5), ("oracle_cmp_dist4", 6)):
                f = getattr(lib, name)
                f.argtypes = [fp] * k
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _f32(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def hull2d(x, y, return_iterations: bool = False):
    """Hull vertex indices (int32), counter-clockwise from the lexicographically
    smallest (x, y) vertex.  Raises OracleError on invalid/non-finite input."""
    lib = _load()
    x, y = _f32(x), _f32(y)
    n = x.shape[0]
    out = np.empty(max(n, 1), dtype=np.int32)
    h = ctypes.c_int64(0)
    it = ctypes.c_int64(0)
    rc = lib.oracle_hull2d(_ptr(x), _ptr(y), n, _ptr(out), ctypes.byref(h), ctypes.byref(it))
    if rc != OK:
        raise OracleError(rc, "hull2d")
    res = out[: h.value].copy()
    return (res, it.value) if return_iterations else res


def hull3d(x, y, z, return_iterations: bool = False):
    """Canonical 3D hull: (vertices, faces) where vertices is a sorted int32
    array and faces a list of int32 arrays (CCW from outside, each starting at
    its smallest index, sorted lexicographically).  Raises OracleError with
    code ERR_DEGENERATE when the points do not span 3D."""
    lib = _load()
    x, y, z = _f32(x), _f32(y), _f32(z)
    n = x.shape[0]
    verts = np.empty(max(n, 1), dtype=np.int32)
    foff = np.empty(2 * n + 16, dtype=np.int32)
    fidx = np.empty(6 * n + 16, dtype=np.int32)
    nv, nf, it = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    rc = lib.oracle_hull3d(_ptr(x), _ptr(y), _ptr(z), n, _ptr(verts), ctypes.byref(nv),
                           _ptr(foff), _ptr(fidx), ctypes.byref(nf), ctypes.byref(it))
    if rc != OK:
        raise OracleError(rc, "hull3d")
    faces = [fidx[foff[i]:foff[i + 1]].copy() for i in range(nf.value)]
    res = (verts[: nv.value].copy(), faces)
    return (res, it.value) if return_iterations else res


def hull4d(x, y, z, w, return_iterations: bool = False):
    """Canonical 4D hull: (vertices, facets) where vertices is the sorted
    int32 array of extreme points and facets a list of int32 arrays, each the
    sorted extreme points on one facet (maximal set of boundary points on a
    supporting hyperplane), sorted lexicographically.  Raises OracleError with
    code ERR_DEGENERATE when the points do not span R^4."""
    lib = _load()
    x, y, z, w = _f32(x), _f32(y), _f32(z), _f32(w)
    n = x.shape[0]
    verts = np.empty(max(n, 1), dtype=np.int32)
    fcap, icap = 64 * n + 64, 256 * n + 256
    foff = np.empty(fcap, dtype=np.int32)
    fidx = np.empty(icap, dtype=np.int32)
    nv, nf, it = ctypes.c_int64(0), ctypes.c_int64(0), ctypes.c_int64(0)
    rc = lib.oracle_hull4d(_ptr(x), _ptr(y), _ptr(z), _ptr(w), n, _ptr(verts), ctypes.byref(nv),
                           _ptr(foff), fcap, _ptr(fidx), icap, ctypes.byref(nf),
                           ctypes.byref(it))
    if rc != OK:
        raise OracleError(rc, "hull4d")
    facets = [fidx[foff[i]:foff[i + 1]].copy() for i in range(nf.value)]
    res = (verts[: nv.value].copy(), facets)
    return (res, it.value) if return_iterations else res


def hull3d_csr(x, y, z):
    """Same as hull3d, as (vertices, face_offsets, face_indices) arrays."""
    verts, faces = hull3d(x, y, z)
    off = np.zeros(len(faces) + 1, dtype=np.int32)
    off[1:] = np.cumsum([len(f) for f in faces]) if faces else []
    idx = np.concatenate(faces).astype(np.int32) if faces else np.zeros(0, np.int32)
    return verts, off, idx


def hull3d_batched(x, y, z, off):
    """Hulls of a batch of clouds (cloud c = points off[c]..off[c+1]): a plain
    loop of hull3d over the clouds.  Returns a list of (status, vertices,
    faces) with global point indices; status is OK, ERR_DEGENERATE or
    ERR_NONFINITE (then no vertices or faces); an empty cloud is OK with no
    faces."""
    x, y, z = _f32(x), _f32(y), _f32(z)
    out = []
    for c in range(len(off) - 1):
        a, b = int(off[c]), int(off[c + 1])
        if a == b:
            out.append((OK, np.zeros(0, np.int32), []))
            continue
        try:
            v, f = hull3d(x[a:b], y[a:b], z[a:b])
        except OracleError as e:
            out.append((e.code, np.zeros(0, np.int32), []))
            continue
        out.append((OK, (v + a).astype(np.int32), [(t + a).astype(np.int32) for t in f]))
    return out


def select(v, off, k):
    """Index of the element of rank k[c] in every segment c: the plain
    definition (sort each segment by (value, index), take position k[c]),
    values ordered by their float32 bit patterns like numbers (-0 before +0,
    NaNs at the ends)."""
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float32))
    u = v.view(np.uint32).astype(np.uint64)
    key = np.where(u & 0x80000000, (~u) & 0xFFFFFFFF, u | 0x80000000)
    out = np.empty(len(off) - 1, dtype=np.int32)
    for c in range(len(off) - 1):
        a, b = int(off[c]), int(off[c + 1])
        idx = np.arange(a, b)
        order = np.lexsort((idx, key[a:b]))
        out[c] = idx[order[int(k[c])]]
    return out


def _pt(p) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(p, dtype=np.float64))


def orient2d(a, b, c) -> int:
    """Exact sign of orient2d: +1 when a, b, c turn counter-clockwise."""
    return _load().oracle_orient2d(*(_ptr(_pt(v)) for v in (a, b, c)))


def cmp_dist2(a, b, p1, p2) -> int:
    """Exact sign of orient2d(a,b,p1) - orient2d(a,b,p2)."""
    return _load().oracle_cmp_dist2(*(_ptr(_pt(v)) for v in (a, b, p1, p2)))


def orient3d(a, b, c, p) -> int:
    """Exact sign of det[b-a; c-a; p-a]."""
    return _load().oracle_orient3d(*(_ptr(_pt(v)) for v in (a, b, c, p)))


def orient4(a, b, c, d, p) -> int:
    """Exact sign of det[b-a; c-a; d-a; p-a] (points as 4 float32 values)."""
    return _load().oracle_orient4(*(_ptr(_pt(q)) for q in (a, b, c, d, p)))


def cmp_dist4(a, b, c, d, p1, p2) -> int:
    """Exact sign of orient4 at p1 minus orient4 at p2."""
    return _load().oracle_cmp_dist4(*(_ptr(_pt(q)) for q in (a, b, c, d, p1, p2)))


def cmp_dist3(a, b, c, p1, p2) -> int:
    """Exact sign of det[b-a; c-a; p1-p2]."""
    return _load().oracle_cmp_dist3(*(_ptr(_pt(v)) for v in (a, b, c, p1, p2)))
