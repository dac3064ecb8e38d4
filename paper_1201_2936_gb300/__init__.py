"""GB300-native segmented Quickhull (Tzeng & Owens, "Finding Convex Hulls
Using Quickhull on the GPU"): Python binding of libqh.

Every step of the hull runs in the CUDA library (include/qh.h); this module
only marshals PyTorch tensors (device memory, streams) into the C ABI.
"""
from __future__ import annotations

import ctypes
from typing import Optional, Tuple, Union

import torch

from . import _native
from ._native import QhOpts, QhResult, RESULT_BYTES

__all__ = ["QHError", "hull2d", "hull2d_async", "workspace_bytes_2d", "Workspace", "hull3d",
           "hull3d_batched", "Hull3DBatch", "workspace_bytes_3d", "workspace_bytes_3d_batched",
           "make_opts", "status_str", "version", "RESULT_BYTES", "result_from_tensor",
           "Hull2DBatch", "hull2d_batched", "workspace_bytes_2d_batched", "hull_measures_2d",
           "hull_measures_3d", "flag_permute", "compact", "select"]

PRED = {"f32": 0, "f64": 1}
LOOP = {"persistent": 0, "host": 1}


class QHError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        super().__init__(f"{what}: {status_str(status)}" if what else status_str(status))
        self.status = status


def status_str(s: int) -> str:
    return _native.lib().qh_status_str(int(s)).decode()


def version() -> str:
    return _native.lib().qh_version().decode()


def make_opts(pred: str = "f32", loop: str = "persistent", blocks_per_sm: int = 0,
              max_iters: int = 0, wait_ns: int = 0, block: int = 0, items: int = 0,
              max_ctas: int = 0, test_hold: int = 0, small_cloud: int = 0,
              max_facets: int = 0) -> QhOpts:
    o = QhOpts()
    _native.lib().qh_default_opts(ctypes.byref(o))
    o.pred_mode = PRED[pred]
    o.loop_mode = LOOP[loop]
    o.blocks_per_sm = blocks_per_sm
    o.max_iters = max_iters
    o.wait_ns = wait_ns
    o.block = block
    o.items = items
    o.max_ctas = max_ctas
    o.test_hold = test_hold
    o.small_cloud = small_cloud
    o.max_facets = max_facets
    return o


def workspace_bytes_2d(n: int, opts: Optional[QhOpts] = None) -> int:
    return int(_native.lib().qh_workspace_bytes_2d(int(n), ctypes.byref(opts) if opts else None))


class Workspace:
    """Device workspace owned by PyTorch's allocator, grown on demand."""

    def __init__(self, device=None):
        self.device = torch.device(device if device is not None else "cuda")
        self.buf: Optional[torch.Tensor] = None

    def get(self, nbytes: int) -> torch.Tensor:
        if self.buf is None or self.buf.numel() < nbytes:
            self.buf = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self.buf


def _stream_handle(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _points_2d(x: torch.Tensor, y: Optional[torch.Tensor]) -> Tuple[int, int, int, int, torch.device]:
    """Return (x_ptr, y_ptr, n, stride, device) for [n,2], [2,n] or separate x, y."""
    if y is None:
        t = x
        if t.dtype != torch.float32 or not t.is_cuda or t.dim() != 2:
            raise ValueError("points must be a CUDA float32 tensor of shape [n, 2] or [2, n]")
        if t.shape[1] == 2 and t.stride(1) == 1 and (t.shape[0] <= 1 or t.stride(0) == 2):
            return t.data_ptr(), t.data_ptr() + 4, t.shape[0], 2, t.device
        if t.shape[0] == 2 and t.stride(1) == 1:
            return t[0].data_ptr(), t[1].data_ptr(), t.shape[1], 1, t.device
        raise ValueError("points must be contiguous [n, 2] or row-contiguous [2, n]")
    for t in (x, y):
        if t.dtype != torch.float32 or not t.is_cuda or t.dim() != 1 or \
                (t.numel() > 1 and t.stride(0) != 1):
            raise ValueError("x and y must be contiguous 1-D CUDA float32 tensors")
    if x.shape != y.shape or x.device != y.device:
        raise ValueError("x and y must have the same length and device")
    return x.data_ptr(), y.data_ptr(), x.shape[0], 1, x.device


def hull2d_async(x: torch.Tensor, y: Optional[torch.Tensor], out: torch.Tensor,
                 result: torch.Tensor, workspace: Workspace, opts: Optional[QhOpts] = None,
                 stream=None) -> None:
    """Launch the hull without synchronising.  `out` is an int32 CUDA tensor
    of at least max(n, 1) entries, `result` a uint8 CUDA tensor of
    RESULT_BYTES bytes that receives the qh_result record."""
    xp, yp, n, stride, dev = _points_2d(x, y)
    o = opts if opts is not None else make_opts()
    nb = workspace_bytes_2d(n, o)
    ws = workspace.get(nb)
    st = _native.lib().qh_hull2d_async(xp, yp, n, stride, out.data_ptr(), result.data_ptr(),
                                       ws.data_ptr(), ws.numel(), ctypes.byref(o),
                                       _stream_handle(stream))
    if st != 0:
        raise QHError(st, "qh_hull2d_async")


MAX_CLOUDS_2D = 8


def _multi_args(clouds, outs):
    """Host arrays of the clouds' device pointers, sizes and strides."""
    k = len(clouds)
    if not 1 <= k <= MAX_CLOUDS_2D:
        raise ValueError(f"between 1 and {MAX_CLOUDS_2D} clouds")
    xs, ys, ns, ss = [], [], [], []
    for c in clouds:
        xp, yp, n, stride, _ = _points_2d(*c) if isinstance(c, tuple) else _points_2d(c, None)
        xs.append(xp)
        ys.append(yp)
        ns.append(n)
        ss.append(stride)
    P = ctypes.c_void_p * k
    I = ctypes.c_int64 * k
    return (k, P(*xs), P(*ys), I(*ns), I(*ss), P(*[o.data_ptr() for o in outs]), ns)


def workspace_bytes_2d_multi(ns, opts: Optional[QhOpts] = None) -> int:
    I = ctypes.c_int64 * len(ns)
    return int(_native.lib().qh_workspace_bytes_2d_multi(len(ns), I(*ns),
                                                         ctypes.byref(opts) if opts else None))


def hull2d_multi_async(clouds, outs, results: torch.Tensor, workspace: Workspace,
                       opts: Optional[QhOpts] = None, stream=None) -> None:
    """Hulls of several 2D clouds in one persistent launch, without
    synchronising.  `clouds`: up to MAX_CLOUDS_2D CUDA float32 tensors ([n, 2],
    [2, n]) or (x, y) pairs; `outs`: one int32 CUDA tensor of at least
    max(n, 1) entries per cloud; `results`: a uint8 CUDA tensor of
    len(clouds) * RESULT_BYTES bytes for the per-cloud qh_result records."""
    k, xs, ys, ns, ss, ps, nl = _multi_args(clouds, outs)
    o = opts if opts is not None else make_opts()
    ws = workspace.get(workspace_bytes_2d_multi(nl, o))
    st = _native.lib().qh_hull2d_multi_async(k, xs, ys, ns, ss, ps, results.data_ptr(),
                                             ws.data_ptr(), ws.numel(), ctypes.byref(o),
                                             _stream_handle(stream))
    if st != 0:
        raise QHError(st, "qh_hull2d_multi_async")


def hull2d_multi(clouds, *, pred: str = "f32", workspace: Optional[Workspace] = None,
                 stream=None, opts: Optional[QhOpts] = None, return_results: bool = False):
    """Hulls of several 2D clouds in one persistent launch (each as hull2d).
    Returns a list of int32 CUDA index tensors (and the result records).
    `opts` (make_opts) replaces the defaults built from `pred`."""
    if not clouds:
        return ([], []) if return_results else []
    first = clouds[0][0] if isinstance(clouds[0], tuple) else clouds[0]
    dev = first.device
    sizes = [(_points_2d(*c) if isinstance(c, tuple) else _points_2d(c, None))[2] for c in clouds]
    outs = [torch.empty(max(n, 1), dtype=torch.int32, device=dev) for n in sizes]
    k, xs, ys, ns, ss, ps, nl = _multi_args(clouds, outs)
    o = opts if opts is not None else make_opts(pred, "persistent")
    if workspace is None:
        workspace = _default_ws.setdefault(str(dev), Workspace(dev))
    ws = workspace.get(workspace_bytes_2d_multi(nl, o))
    counts = (ctypes.c_int64 * k)()
    res = (QhResult * k)()
    st = _native.lib().qh_hull2d_multi(k, xs, ys, ns, ss, ps, counts, res, ws.data_ptr(),
                                       ws.numel(), ctypes.byref(o), _stream_handle(stream))
    if st not in (0, 2):  # a non-finite cloud is reported in its own record
        raise QHError(st, "qh_hull2d_multi")
    out = [outs[c][: counts[c]] for c in range(k)]
    return (out, [res[c].as_dict() for c in range(k)]) if return_results else out


def debug_timeline_2d(workspace: Workspace, n: int, stream=None):
    """Per-iteration rows (iteration, live points, segments, pass ns, update ns)
    of the last persistent-loop 2D call on `workspace` with n points."""
    import numpy as np
    rows = np.zeros((64, 5), dtype=np.int64)
    nr = ctypes.c_int32(0)
    st = _native.lib().qh_debug_timeline_2d(workspace.buf.data_ptr(), int(n),
                                            rows.ctypes.data_as(ctypes.c_void_p), 64,
                                            ctypes.byref(nr), _stream_handle(stream))
    if st != 0:
        raise QHError(st, "qh_debug_timeline_2d")
    return rows[: nr.value]


def debug_phases_3d(ws: torch.Tensor, stream=None):
    """Device ns of the last 3D call on the workspace tensor `ws`: initial
    simplex, first assignment, its table, its scatter + certify + exact, and
    the whole persistent kernel."""
    import numpy as np
    out = np.zeros(5, dtype=np.int64)
    st = _native.lib().qh_debug_phases_3d(ws.data_ptr(), out.ctypes.data_as(ctypes.c_void_p),
                                          _stream_handle(stream))
    if st != 0:
        raise QHError(st, "qh_debug_phases_3d")
    return out


def workspace_bytes_3d(n: int, opts: Optional[QhOpts] = None) -> int:
    return int(_native.lib().qh_workspace_bytes_3d(int(n), ctypes.byref(opts) if opts else None))


def _points_3d(x, y, z):
    if y is None and z is None:
        t = x
        if t.dtype != torch.float32 or not t.is_cuda or t.dim() != 2:
            raise ValueError("points must be a CUDA float32 tensor of shape [n, 3] or [3, n]")
        if t.shape[1] == 3 and t.stride(1) == 1 and (t.shape[0] <= 1 or t.stride(0) == 3):
            p = t.data_ptr()
            return p, p + 4, p + 8, t.shape[0], 3, t.device
        if t.shape[0] == 3 and t.stride(1) == 1:
            return t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(), t.shape[1], 1, t.device
        raise ValueError("points must be contiguous [n, 3] or row-contiguous [3, n]")
    for t in (x, y, z):
        if t.dtype != torch.float32 or not t.is_cuda or t.dim() != 1 or \
                (t.numel() > 1 and t.stride(0) != 1):
            raise ValueError("x, y, z must be contiguous 1-D CUDA float32 tensors")
    if not (x.shape == y.shape == z.shape):
        raise ValueError("x, y, z must have the same length")
    return x.data_ptr(), y.data_ptr(), z.data_ptr(), x.shape[0], 1, x.device


def hull3d(x: torch.Tensor, y: Optional[torch.Tensor] = None, z: Optional[torch.Tensor] = None,
           *, pred: str = "f32", workspace: Optional[Workspace] = None, stream=None,
           opts: Optional[QhOpts] = None, return_result: bool = False):
    """Convex hull of 3D float32 points on the GPU.

    Returns (vertices, face_offsets, face_indices) as int32 CUDA tensors:
    sorted vertex indices and the faces as CSR polygons (maximal coplanar
    faces, counter-clockwise from outside, starting at their smallest index,
    sorted lexicographically).  Points are [n, 3], [3, n] or x, y, z.
    `opts` (make_opts: launch shape, limits) replaces the defaults built from
    `pred`."""
    xp, yp, zp, n, stride, dev = _points_3d(x, y, z)
    o = opts if opts is not None else make_opts(pred, "persistent")
    if workspace is None:
        workspace = _default_ws.setdefault(str(dev), Workspace(dev))
    ws = workspace.get(workspace_bytes_3d(n, o))
    verts = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    foff = torch.empty(2 * n + 2, dtype=torch.int32, device=dev)
    fidx = torch.empty(max(6 * n, 1), dtype=torch.int32, device=dev)
    nv, nf = ctypes.c_int64(0), ctypes.c_int64(0)
    res = QhResult()
    st = _native.lib().qh_hull3d(xp, yp, zp, n, stride, verts.data_ptr(), ctypes.byref(nv),
                                 foff.data_ptr(), fidx.data_ptr(), ctypes.byref(nf),
                                 ctypes.byref(res), ws.data_ptr(), ws.numel(), ctypes.byref(o),
                                 _stream_handle(stream))
    if st != 0:
        raise QHError(st, "qh_hull3d")
    off = foff[: nf.value + 1] if nf.value > 0 else foff[:1].zero_()
    out = (verts[: nv.value], off, fidx[: int(res.extra[2])])
    return (out, res.as_dict()) if return_result else out


def workspace_bytes_4d(n: int, opts: Optional[QhOpts] = None) -> int:
    return int(_native.lib().qh_workspace_bytes_4d(int(n), ctypes.byref(opts) if opts else None))


def hull4d(x: torch.Tensor, y: Optional[torch.Tensor] = None, z: Optional[torch.Tensor] = None,
           w: Optional[torch.Tensor] = None, *, workspace: Optional[Workspace] = None,
           stream=None, opts: Optional[QhOpts] = None, return_result: bool = False):
    """Convex hull of 4D float32 points on the GPU (qh_hull4d).

    Returns (vertices, facet_offsets, facet_indices) as int32 CUDA tensors:
    the sorted extreme points and, as CSR lists, every facet's sorted extreme
    points, facets in lexicographic order.  Points are a [n, 4] tensor, a
    [4, n] tensor, or x, y, z, w."""
    if y is None and z is None and w is None:
        t = x
        if t.dtype != torch.float32 or not t.is_cuda or t.dim() != 2:
            raise ValueError("points must be a CUDA float32 tensor of shape [n, 4] or [4, n]")
        if t.shape[1] == 4 and t.stride(1) == 1 and (t.shape[0] <= 1 or t.stride(0) == 4):
            p = t.data_ptr()
            xp, yp, zp, wp, n, stride = p, p + 4, p + 8, p + 12, t.shape[0], 4
        elif t.shape[0] == 4 and t.stride(1) == 1:
            xp, yp, zp, wp, n, stride = (t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr(),
                                         t[3].data_ptr(), t.shape[1], 1)
        else:
            raise ValueError("points must be contiguous [n, 4] or row-contiguous [4, n]")
        dev = t.device
    else:
        for c in (x, y, z, w):
            if c is None or c.dtype != torch.float32 or not c.is_cuda or c.dim() != 1 or \
                    (c.numel() > 1 and c.stride(0) != 1):
                raise ValueError("x, y, z, w must be contiguous 1-D CUDA float32 tensors")
        if not (x.shape == y.shape == z.shape == w.shape):
            raise ValueError("x, y, z, w must have the same length")
        xp, yp, zp, wp, n, stride = (x.data_ptr(), y.data_ptr(), z.data_ptr(), w.data_ptr(),
                                     x.shape[0], 1)
        dev = x.device
    o = opts if opts is not None else make_opts("f32", "persistent")
    if workspace is None:
        workspace = _default_ws.setdefault(str(dev), Workspace(dev))
    nb = workspace_bytes_4d(n, o)
    if nb == 0:
        raise QHError(1, "qh_workspace_bytes_4d")
    ws = workspace.get(nb)
    verts = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    cap_f, cap_i = 8 * n + 64, 32 * n + 256
    for _ in range(2):
        foff = torch.empty(cap_f + 1, dtype=torch.int32, device=dev)
        fidx = torch.empty(cap_i, dtype=torch.int32, device=dev)
        nv, nf = ctypes.c_int64(0), ctypes.c_int64(0)
        res = QhResult()
        st = _native.lib().qh_hull4d(xp, yp, zp, wp, n, stride, verts.data_ptr(), ctypes.byref(nv),
                                     foff.data_ptr(), cap_f, fidx.data_ptr(), cap_i,
                                     ctypes.byref(nf), ctypes.byref(res), ws.data_ptr(),
                                     ws.numel(), ctypes.byref(o), _stream_handle(stream))
        if st == 5 and (nf.value > cap_f or res.extra[2] > cap_i):  # QH_ERR_CAPACITY: grow once
            cap_f, cap_i = max(cap_f, nf.value), max(cap_i, int(res.extra[2]))
            continue
        break
    if st != 0:
        raise QHError(st, "qh_hull4d")
    out = (verts[: nv.value], foff[: nf.value + 1], fidx[: int(res.extra[2])])
    return (out, res.as_dict()) if return_result else out


def debug_timeline_4d():
    """Per-iteration rows of the last hull4d call on this thread: iteration,
    segments, live points, apexes of the previous iteration, uncertified
    apexes, host ns, candidates claiming in rounds 0-2 of the previous
    iteration."""
    import numpy as np
    rows = np.zeros((4096, 9), dtype=np.int64)
    nr = ctypes.c_int32(0)
    st = _native.lib().qh_debug_timeline_4d(rows.ctypes.data_as(ctypes.c_void_p), 4096,
                                            ctypes.byref(nr))
    if st != 0:
        raise QHError(st, "qh_debug_timeline_4d")
    return rows[: nr.value]


DEBUG_SITES = {1: "bulk copy alignment", 2: "mbarrier alignment", 3: "bulk copy source range",
               4: "point scatter destination", 5: "segment index", 6: "hull slot",
               7: "vector load alignment"}


def debug_checks(reset: bool = False) -> dict:
    """qh_debug_checks: the device-side check record of a library built with
    QH_DEBUG_BUILD=1 (failed checks, first site and its values).  Raises
    QHError(QH_ERR_NOT_SUPPORTED) on the default build."""
    rec = _native.QhDebugRecord()
    st = _native.lib().qh_debug_checks(ctypes.byref(rec), 1 if reset else 0)
    if st != 0:
        raise QHError(st, "qh_debug_checks")
    return {"failures": rec.failures, "site": DEBUG_SITES.get(rec.site, rec.site),
            "a": rec.a, "b": rec.b, "enabled": bool(rec.enabled)}


NOALLOC_MAX_POINTS = 131072


def hull2d_noalloc(x: torch.Tensor, y: Optional[torch.Tensor] = None, *,
                   out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """qh_hull2d_noalloc: the 2D hull with the library's fixed device scratch
    (no workspace; n <= NOALLOC_MAX_POINTS).  For callers that cannot
    allocate device memory while they run; calls on one device must not
    overlap."""
    xp, yp, n, stride, dev = _points_2d(x, y)
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    cnt = ctypes.c_int64(0)
    st = _native.lib().qh_hull2d_noalloc(xp, yp, n, stride, out.data_ptr(), ctypes.byref(cnt),
                                         _stream_handle(stream))
    if st != 0:
        raise QHError(st, "qh_hull2d_noalloc")
    return out[: cnt.value]


def debug_timeline_3d(workspace: Workspace, n: int, stream=None):
    """Per-iteration rows of the last 3D call on `workspace` with n points:
    iteration, live points, segments, apexes, then ns of select, rounds,
    assign, table, scatter, exact."""
    import numpy as np
    rows = np.zeros((64, 10), dtype=np.int64)
    nr = ctypes.c_int32(0)
    st = _native.lib().qh_debug_timeline_3d(workspace.buf.data_ptr(), int(n),
                                            rows.ctypes.data_as(ctypes.c_void_p), 64,
                                            ctypes.byref(nr), _stream_handle(stream))
    if st != 0:
        raise QHError(st, "qh_debug_timeline_3d")
    return rows[: nr.value]


def result_from_tensor(result: torch.Tensor) -> QhResult:
    raw = bytes(result.cpu().numpy().tobytes())
    return QhResult.from_buffer_copy(raw[:RESULT_BYTES])


_default_ws = {}


def hull2d(x: torch.Tensor, y: Optional[torch.Tensor] = None, *, pred: str = "f32",
           loop: str = "persistent", workspace: Optional[Workspace] = None,
           out: Optional[torch.Tensor] = None, stream=None, opts: Optional[QhOpts] = None,
           return_result: bool = False) -> Union[torch.Tensor, Tuple[torch.Tensor, dict]]:
    """Convex hull of 2D float32 points on the GPU.

    Returns an int32 CUDA tensor with the hull vertex indices in counter-
    clockwise order from the lexicographically smallest (x, y) vertex.
    Points are a [n, 2] tensor, a [2, n] tensor, or separate x and y.
    `opts` (make_opts) overrides pred and loop.
    """
    xp, yp, n, stride, dev = _points_2d(x, y)
    o = opts if opts is not None else make_opts(pred, loop)
    if workspace is None:
        workspace = _default_ws.setdefault(str(dev), Workspace(dev))
    ws = workspace.get(workspace_bytes_2d(n, o))
    if out is None:
        out = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    cnt = ctypes.c_int64(0)
    res = QhResult()
    st = _native.lib().qh_hull2d(xp, yp, n, stride, out.data_ptr(), ctypes.byref(cnt),
                                 ctypes.byref(res), ws.data_ptr(), ws.numel(), ctypes.byref(o),
                                 _stream_handle(stream))
    if st != 0:
        raise QHError(st, "qh_hull2d")
    idx = out[: cnt.value]
    return (idx, res.as_dict()) if return_result else idx


# ---------------------------------------------------------------------- batched 3D
def workspace_bytes_3d_batched(n: int, ncloud: int, opts: Optional[QhOpts] = None) -> int:
    return int(_native.lib().qh_workspace_bytes_3d_batched(int(n), int(ncloud),
                                                           ctypes.byref(opts) if opts else None))


class Hull3DBatch:
    """Hulls of a batch of 3D clouds (qh_hull3d_batched) with every output
    buffer allocated once, so that one call can be captured in a CUDA graph
    and replayed.  Points: [n, 3], [3, n] or x, y, z CUDA float32; cloud_off:
    int64 CUDA tensor [ncloud + 1] (CSR offsets).  Output indices are global
    (into the concatenated points)."""

    def __init__(self, x, y=None, z=None, cloud_off: torch.Tensor = None, *, pred: str = "f32",
                 opts: Optional[QhOpts] = None):
        if cloud_off is None or cloud_off.dtype != torch.int64 or not cloud_off.is_cuda or \
                cloud_off.dim() != 1 or cloud_off.numel() < 2:
            raise ValueError("cloud_off must be a CUDA int64 tensor of ncloud + 1 offsets")
        self._inputs = (x, y, z, cloud_off.contiguous())
        self.xp, self.yp, self.zp, self.n, self.stride, dev = _points_3d(x, y, z)
        self.cloud_off = self._inputs[3]
        self.ncloud = cloud_off.numel() - 1
        self.opts = opts if opts is not None else make_opts(pred)
        n, nc = self.n, self.ncloud
        i32 = dict(dtype=torch.int32, device=dev)
        self.verts = torch.empty(max(n, 1), **i32)
        self.cloud_voff = torch.empty(nc + 1, **i32)
        self.face_off = torch.empty(2 * n + 1, **i32)
        self.face_idx = torch.empty(max(6 * n, 1), **i32)
        self.cloud_foff = torch.empty(nc + 1, **i32)
        self.cloud_status = torch.empty(nc, **i32)
        self.result = torch.zeros(RESULT_BYTES, dtype=torch.uint8, device=dev)
        nb = workspace_bytes_3d_batched(n, nc, self.opts)
        if nb == 0:
            raise QHError(1, "qh_workspace_bytes_3d_batched")
        self.ws = torch.empty(nb, dtype=torch.uint8, device=dev)
        self.graph = None

    def _args(self):
        return (self.xp, self.yp, self.zp, self.stride, self.cloud_off.data_ptr(), self.ncloud,
                self.n, self.verts.data_ptr(), self.cloud_voff.data_ptr(),
                self.face_off.data_ptr(), self.face_idx.data_ptr(), self.cloud_foff.data_ptr(),
                self.cloud_status.data_ptr(), self.result.data_ptr(), self.ws.data_ptr(),
                self.ws.numel())

    def enqueue(self, stream=None) -> None:
        """Issue the whole batch on the stream (no synchronisation)."""
        st = _native.lib().qh_hull3d_batched(*self._args(), ctypes.byref(self.opts),
                                             _stream_handle(stream))
        if st != 0:
            raise QHError(st, "qh_hull3d_batched")

    def tune(self, reps: int = 3, stream=None):
        """Autotune the launch on this batch (qh_autotune_3d_batched): the
        shape, then the small-cloud threshold at the fastest shape; keeps the
        fastest in self.opts and returns [(block, items, ctas_per_sm,
        small_cloud, ms), ...]."""
        import numpy as np
        best = QhOpts()
        ctypes.memmove(ctypes.byref(best), ctypes.byref(self.opts), ctypes.sizeof(QhOpts))
        ms = np.zeros(64, dtype=np.float32)
        shape = np.zeros(4 * 64, dtype=np.int32)
        nc = ctypes.c_int32(0)
        st = _native.lib().qh_autotune_3d_batched(
            *self._args(), int(reps), ctypes.byref(best), ms.ctypes.data_as(ctypes.c_void_p),
            shape.ctypes.data_as(ctypes.c_void_p), 64, ctypes.byref(nc), _stream_handle(stream))
        if st != 0:
            raise QHError(st, "qh_autotune_3d_batched")
        self.opts = best
        return [(int(shape[4 * i]), int(shape[4 * i + 1]), int(shape[4 * i + 2]),
                 int(shape[4 * i + 3]), float(ms[i])) for i in range(nc.value)]

    def capture(self) -> None:
        """Capture one enqueue() in a CUDA graph (after a warm-up run)."""
        s = torch.cuda.Stream(device=self.verts.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.enqueue()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.enqueue()
        self.graph = g

    def replay(self) -> None:
        self.graph.replay()

    def result_dict(self) -> dict:
        r = result_from_tensor(self.result)
        return r.as_dict()

    def measures(self, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """[ncloud, 2] float64 (surface area, volume) of the hulls of the last
        run (qh_measures3d, asynchronous)."""
        if out is None:
            out = torch.empty(self.ncloud, 2, dtype=torch.float64, device=self.verts.device)
        st = _native.lib().qh_measures3d(self.xp, self.yp, self.zp, self.stride, self.ncloud,
                                         self.face_off.data_ptr(), self.face_idx.data_ptr(),
                                         self.cloud_foff.data_ptr(), out.data_ptr(),
                                         _stream_handle(stream))
        if st != 0:
            raise QHError(st, "qh_measures3d")
        return out

    def backward(self, grad_meas: torch.Tensor, grad: torch.Tensor, stream=None) -> torch.Tensor:
        """dL/dpoints into `grad` (float32, same layout as the points) from
        dL/d(area, volume) [ncloud, 2] float64 (qh_hull3d_backward)."""
        (gx, gy, gz), _, gstride = _rows(grad, 3)
        if getattr(self, "_scratch", None) is None:
            self._scratch = torch.empty(3 * max(self.n, 1), dtype=torch.float64,
                                        device=self.verts.device)
        st = _native.lib().qh_hull3d_backward(self.xp, self.yp, self.zp, self.stride,
                                              self.ncloud, self.n, self.face_off.data_ptr(),
                                              self.face_idx.data_ptr(), self.cloud_foff.data_ptr(),
                                              grad_meas.data_ptr(), gx, gy, gz, gstride,
                                              self._scratch.data_ptr(), _stream_handle(stream))
        if st != 0:
            raise QHError(st, "qh_hull3d_backward")
        return grad

    def outputs(self):
        """(verts, cloud_vert_off, face_off, face_idx, cloud_face_off,
        cloud_status) after the last run, sliced to their lengths
        (synchronises).  Raises QHError if the call failed."""
        r = result_from_tensor(self.result)
        if r.status != 0:
            raise QHError(r.status, "qh_hull3d_batched")
        nv, nf, ni = int(r.extra[0]), int(r.extra[1]), int(r.extra[2])
        return (self.verts[:nv], self.cloud_voff, self.face_off[: nf + 1], self.face_idx[:ni],
                self.cloud_foff, self.cloud_status)


def hull3d_batched(x, y=None, z=None, cloud_off: torch.Tensor = None, *, pred: str = "f32",
                   opts: Optional[QhOpts] = None):
    """One batched call (see Hull3DBatch.outputs for the returned tuple)."""
    b = Hull3DBatch(x, y, z, cloud_off, pred=pred, opts=opts)
    b.enqueue()
    return b.outputs()


# ---------------------------------------------------------------------- batched 2D
def workspace_bytes_2d_batched(n: int, ncloud: int, opts: Optional[QhOpts] = None) -> int:
    return int(_native.lib().qh_workspace_bytes_2d_batched(int(n), int(ncloud),
                                                           ctypes.byref(opts) if opts else None))


def _check_off(cloud_off):
    if cloud_off is None or cloud_off.dtype != torch.int64 or not cloud_off.is_cuda or \
            cloud_off.dim() != 1 or cloud_off.numel() < 2 or \
            (cloud_off.numel() > 1 and cloud_off.stride(0) != 1):
        raise ValueError("cloud_off must be a contiguous CUDA int64 tensor of ncloud + 1 offsets")


class Hull2DBatch:
    """Hulls of a batch of 2D clouds (qh_hull2d_batched), output buffers
    allocated once (graph-capturable).  Points [n, 2], [2, n] or x, y CUDA
    float32; cloud_off int64 CUDA [ncloud + 1].  Cloud c's hull (global
    indices) is out[cloud_off[c] : cloud_off[c] + count[c]]."""

    def __init__(self, x, y=None, cloud_off: torch.Tensor = None, *, pred: str = "f32",
                 opts: Optional[QhOpts] = None, workspace: Optional[Workspace] = None):
        _check_off(cloud_off)
        self._inputs = (x, y, cloud_off)
        self.xp, self.yp, self.n, self.stride, dev = _points_2d(x, y)
        self.cloud_off = cloud_off
        self.ncloud = cloud_off.numel() - 1
        self.opts = opts if opts is not None else make_opts(pred)
        i32 = dict(dtype=torch.int32, device=dev)
        self.out = torch.empty(max(self.n, 1), **i32)
        self.count = torch.empty(self.ncloud, **i32)
        self.status = torch.empty(self.ncloud, **i32)
        self.result = torch.zeros(RESULT_BYTES, dtype=torch.uint8, device=dev)
        nb = workspace_bytes_2d_batched(self.n, self.ncloud, self.opts)
        if nb == 0:
            raise QHError(1, "qh_workspace_bytes_2d_batched")
        self.ws = (workspace or Workspace(dev)).get(nb)
        self.graph = None

    def enqueue(self, stream=None) -> None:
        st = _native.lib().qh_hull2d_batched(
            self.xp, self.yp, self.stride, self.cloud_off.data_ptr(), self.ncloud, self.n,
            self.out.data_ptr(), self.count.data_ptr(), self.status.data_ptr(),
            self.result.data_ptr(), self.ws.data_ptr(), self.ws.numel(), ctypes.byref(self.opts),
            _stream_handle(stream))
        if st != 0:
            raise QHError(st, "qh_hull2d_batched")

    def capture(self) -> None:
        s = torch.cuda.Stream(device=self.out.device)
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.enqueue()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.enqueue()
        self.graph = g

    def replay(self) -> None:
        self.graph.replay()

    def result_dict(self) -> dict:
        return result_from_tensor(self.result).as_dict()

    def measures(self, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """[ncloud, 2] float64 (perimeter, area) of the hulls of the last run
        (qh_measures2d, asynchronous)."""
        if out is None:
            out = torch.empty(self.ncloud, 2, dtype=torch.float64, device=self.out.device)
        st = _native.lib().qh_measures2d(self.xp, self.yp, self.stride, self.cloud_off.data_ptr(),
                                         self.ncloud, self.out.data_ptr(), self.count.data_ptr(),
                                         out.data_ptr(), _stream_handle(stream))
        if st != 0:
            raise QHError(st, "qh_measures2d")
        return out

    def backward(self, grad_meas: torch.Tensor, grad: torch.Tensor, stream=None) -> torch.Tensor:
        """dL/dpoints into `grad` (float32, same layout as the points) from
        dL/d(perimeter, area) [ncloud, 2] float64 (qh_hull2d_backward)."""
        (gx, gy), _, gstride = _rows(grad, 2)
        st = _native.lib().qh_hull2d_backward(self.xp, self.yp, self.stride,
                                              self.cloud_off.data_ptr(), self.ncloud, self.n,
                                              self.out.data_ptr(), self.count.data_ptr(),
                                              grad_meas.data_ptr(), gx, gy, gstride,
                                              _stream_handle(stream))
        if st != 0:
            raise QHError(st, "qh_hull2d_backward")
        return grad

    def outputs(self):
        """(out, count, status) after the last run (synchronises); raises
        QHError if the call failed."""
        r = result_from_tensor(self.result)
        if r.status != 0:
            raise QHError(r.status, "qh_hull2d_batched")
        return self.out, self.count, self.status


def hull2d_batched(x, y=None, cloud_off: torch.Tensor = None, *, pred: str = "f32",
                   opts: Optional[QhOpts] = None):
    """One batched 2D call: (out, count, status), see Hull2DBatch."""
    b = Hull2DBatch(x, y, cloud_off, pred=pred, opts=opts)
    b.enqueue()
    return b.outputs()


# ---------------------------------------------------------------------- differentiable measures
def _rows(pts: torch.Tensor, d: int):
    """[d, n] row-contiguous or [n, d] contiguous float32 CUDA -> (row pointers, n, stride)."""
    if pts.dtype != torch.float32 or not pts.is_cuda or pts.dim() != 2:
        raise ValueError(f"points must be a CUDA float32 tensor [{d}, n] or [n, {d}]")
    if pts.shape[0] == d and pts.stride(1) == 1:
        return [pts[i].data_ptr() for i in range(d)], pts.shape[1], 1
    if pts.shape[1] == d and pts.stride(1) == 1 and (pts.shape[0] <= 1 or pts.stride(0) == d):
        return [pts.data_ptr() + 4 * i for i in range(d)], pts.shape[0], d
    raise ValueError(f"points must be row-contiguous [{d}, n] or contiguous [n, {d}]")


class _Measures2D(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pts, cloud_off, pred):
        ws = _default_ws.setdefault(str(pts.device), Workspace(pts.device))
        b = Hull2DBatch(pts.detach(), None, cloud_off, pred=pred, workspace=ws)
        b.enqueue()
        meas = b.measures()
        b.outputs()  # raises on a failed hull
        ctx.batch = b
        return meas

    @staticmethod
    def backward(ctx, gm):
        b = ctx.batch
        g = gm.detach().to(torch.float64).contiguous()
        grad = b.backward(g, torch.empty_like(b._inputs[0]))
        ctx.batch = None
        return grad, None, None


def hull_measures_2d(pts: torch.Tensor, cloud_off: torch.Tensor, *, pred: str = "f32"):
    """[ncloud, 2] float64: (perimeter, area) of each cloud's hull, differentiable
    with respect to pts ([2, n] or [n, 2] CUDA float32; gradient on the hull
    vertices only, computed by qh_hull2d_backward)."""
    _check_off(cloud_off)
    return _Measures2D.apply(pts, cloud_off, pred)


class _Measures3D(torch.autograd.Function):
    @staticmethod
    def forward(ctx, pts, cloud_off, pred):
        b = Hull3DBatch(pts.detach(), None, None, cloud_off, pred=pred)
        b.enqueue()
        meas = b.measures()
        b.outputs()  # raises on a failed hull
        ctx.batch = b
        return meas

    @staticmethod
    def backward(ctx, gm):
        b = ctx.batch
        g = gm.detach().to(torch.float64).contiguous()
        grad = b.backward(g, torch.empty_like(b._inputs[0]))
        ctx.batch = None
        return grad, None, None


def hull_measures_3d(pts: torch.Tensor, cloud_off: torch.Tensor, *, pred: str = "f32"):
    """[ncloud, 2] float64: (surface area, volume) of each cloud's hull,
    differentiable with respect to pts ([3, n] or [n, 3] CUDA float32;
    gradient on the hull vertices only, computed by qh_hull3d_backward)."""
    _check_off(cloud_off)
    return _Measures3D.apply(pts, cloud_off, pred)


# ---------------------------------------------------------------------- segmented primitives
def _i32_cuda(t, name):
    if t.dtype != torch.int32 or not t.is_cuda or t.dim() != 1 or \
            (t.numel() > 1 and t.stride(0) != 1):
        raise ValueError(f"{name} must be a contiguous 1-D CUDA int32 tensor")


def _seg_ws(n: int, nseg: int, dev) -> torch.Tensor:
    nb = int(_native.lib().qh_segmented_workspace_bytes(int(n), int(nseg)))
    if nb == 0:
        raise QHError(1, "qh_segmented_workspace_bytes")
    return _default_ws.setdefault("seg:" + str(dev), Workspace(dev)).get(nb)


def flag_permute(f: torch.Tensor, s: torch.Tensor, k: int):
    """k-state flagPermute (Algorithm 2) on the GPU: (p, s_new) as int32
    CUDA tensors (qh_flag_permute)."""
    _i32_cuda(f, "f")
    _i32_cuda(s, "s")
    n = f.numel()
    p = torch.empty(max(n, 1), dtype=torch.int32, device=f.device)
    s_new = torch.empty(max(n, 1), dtype=torch.int32, device=f.device)
    ws = _seg_ws(n, 1, f.device)
    st = _native.lib().qh_flag_permute(f.data_ptr(), s.data_ptr(), n, int(k), p.data_ptr(),
                                       s_new.data_ptr(), ws.data_ptr(), ws.numel(),
                                       _stream_handle(None))
    if st != 0:
        raise QHError(st, "qh_flag_permute")
    return p[:n], s_new[:n]


def compact(b: torch.Tensor, s: torch.Tensor):
    """compact (Algorithm 3) on the GPU: (p, s_new, n_new) (qh_compact)."""
    _i32_cuda(b, "b")
    _i32_cuda(s, "s")
    n = b.numel()
    p = torch.empty(max(n, 1), dtype=torch.int32, device=b.device)
    s_new = torch.empty(max(n, 1), dtype=torch.int32, device=b.device)
    nn = ctypes.c_int64(0)
    ws = _seg_ws(n, 1, b.device)
    st = _native.lib().qh_compact(b.data_ptr(), s.data_ptr(), n, p.data_ptr(), s_new.data_ptr(),
                                  ctypes.byref(nn), ws.data_ptr(), ws.numel(),
                                  _stream_handle(None))
    if st != 0:
        raise QHError(st, "qh_compact")
    return p[:n], s_new[: nn.value], nn.value


def select(v: torch.Tensor, seg_off: torch.Tensor, k: torch.Tensor, return_iters: bool = False,
           loop: str = "device"):
    """Index of the element of rank k[c] in every segment c of v (qh_select):
    v float32 CUDA [n], seg_off int64 CUDA [nseg + 1], k int64 CUDA [nseg].
    loop="device": one persistent launch for all rounds; "host": one host
    iteration per round (qh_select_host_loop)."""
    if loop not in ("device", "host"):
        raise ValueError("loop must be 'device' or 'host'")
    if v.dtype != torch.float32 or not v.is_cuda or v.dim() != 1 or \
            (v.numel() > 1 and v.stride(0) != 1):
        raise ValueError("v must be a contiguous 1-D CUDA float32 tensor")
    _check_off(seg_off)
    if k.dtype != torch.int64 or not k.is_cuda or k.numel() != seg_off.numel() - 1:
        raise ValueError("k must be a CUDA int64 tensor with one rank per segment")
    k = k.contiguous()
    nseg = seg_off.numel() - 1
    out = torch.empty(nseg, dtype=torch.int32, device=v.device)
    it = ctypes.c_int64(0)
    ws = _seg_ws(v.numel(), nseg, v.device)
    fn = _native.lib().qh_select if loop == "device" else _native.lib().qh_select_host_loop
    st = fn(v.data_ptr(), seg_off.data_ptr(), nseg, v.numel(), k.data_ptr(), out.data_ptr(),
            ctypes.byref(it), ws.data_ptr(), ws.numel(), _stream_handle(None))
    if st != 0:
        raise QHError(st, "qh_select")
    return (out, it.value) if return_iters else out
