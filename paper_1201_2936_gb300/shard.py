"""One hull over several ranks (one GPU each).

The hull of a union is the hull of the union of the parts' hulls, so a
cloud split into contiguous shards needs one exchange: every rank hulls its
shard, the shard hulls' vertices (global indices and coordinates) are
all-gathered, and the hull of the gathered vertices is the answer (computed
on every rank).  Only the shard hulls travel: h_g points per rank, small
next to n / G except for points on a circle or sphere.

`hull_fn` computes a hull on one rank's data and returns local indices; by
default it is the library's GPU hull.  In 3D a shard may not span space
(fewer than four points, or all of them coplanar) although the whole cloud
does: hull_fn then returns None and every point of that shard is a
candidate, which keeps the union of the candidates' hull equal to the
cloud's.  The collective is torch.distributed (NCCL between GPUs; the tests
run it with gloo on CPU ranks).
"""
from __future__ import annotations

import ctypes
from typing import Callable, Optional, Sequence, Tuple

import numpy as np
import torch
import torch.distributed as dist


def shard_range(n: int, rank: int, world: int) -> Tuple[int, int]:
    """Contiguous shard [lo, hi) of rank `rank`: sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


QH_ERR_DEGENERATE = 3


def _gpu_hull(coords: Sequence[torch.Tensor]):
    from . import QHError, hull2d, hull3d
    if len(coords) == 2:
        return hull2d(coords[0], coords[1]).long()
    try:
        v, _, _ = hull3d(coords[0], coords[1], coords[2])
    except QHError as e:
        if e.status == QH_ERR_DEGENERATE:
            return None
        raise
    return v.long()


def _degenerate():
    from . import QHError
    return QHError(QH_ERR_DEGENERATE, "sharded hull: the points do not span 3D")


def _candidates(coords: Sequence[torch.Tensor], group, local_fn):
    """This rank's shard hull, all-gathered: the candidates' global indices
    in increasing order (duplicate locations keep their lowest index, as in
    the one-rank hull)."""
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    n = int(coords[0].numel())
    lo, hi = shard_range(n, rank, world)
    local = local_fn([c[lo:hi] for c in coords]) if hi > lo else \
        torch.zeros(0, dtype=torch.long, device=coords[0].device)
    if local is None:  # a shard that does not span 3D: all its points
        local = torch.arange(hi - lo, dtype=torch.long, device=coords[0].device)
    gidx = local.to(torch.long) + lo
    # exchange: sizes first, then the padded index lists
    dev = coords[0].device
    cnt = torch.tensor([gidx.numel()], dtype=torch.long, device=dev)
    if world > 1:
        sizes = [torch.zeros_like(cnt) for _ in range(world)]
        dist.all_gather(sizes, cnt, group=group)
        m = int(max(s.item() for s in sizes))
        pad = torch.full((max(m, 1),), -1, dtype=torch.long, device=dev)
        pad[: gidx.numel()] = gidx
        parts = [torch.empty_like(pad) for _ in range(world)]
        dist.all_gather(parts, pad, group=group)
        cand = torch.cat([p[: int(s.item())] for p, s in zip(parts, sizes)])
    else:
        cand = gidx
    cand, _ = torch.sort(cand)
    return cand


def sharded_hull(coords: Sequence[torch.Tensor], group=None,
                 hull_fn: Optional[Callable] = None):
    """Hull of the whole cloud, whose coordinates every rank holds (1-D
    tensors of the same length n).  Each rank hulls its shard; returns the
    global indices of the final hull as hull_fn orders them (2D: CCW from the
    lexicographic min; 3D: increasing vertex indices) and the gathered
    candidate indices.  sharded_hull3d also returns the 3D faces."""
    hull_fn = hull_fn or _gpu_hull
    cand = _candidates(coords, group, hull_fn)
    sub = hull_fn([c[cand] for c in coords])
    if sub is None:
        raise _degenerate()
    return cand[sub.to(torch.long)], cand


def _gpu_hull3d_faces(coords):
    from . import QHError, hull3d
    try:
        v, off, idx = hull3d(coords[0], coords[1], coords[2])
    except QHError as e:
        if e.status == QH_ERR_DEGENERATE:
            return None
        raise
    return v.long(), off.long(), idx.long()


def sharded_hull3d(coords: Sequence[torch.Tensor], group=None,
                   hull_fn: Optional[Callable] = None):
    """3D hull of the whole cloud over the ranks, with its faces: returns
    (vertices, face_offsets, face_indices) in global indices, equal to the
    one-rank hull's canonical output.  hull_fn(coords) -> (vertices,
    face_offsets, face_indices) of a cloud, or None when its points do not
    span 3D (default: the library's GPU hull).  A whole cloud that does not
    span 3D raises QHError(QH_ERR_DEGENERATE).
    The candidates are in increasing global index, so mapping the final
    hull's candidate-local indices to global ones keeps the canonical order
    (sorted vertices, faces from their smallest index, faces in
    lexicographic order)."""
    hull_fn = hull_fn or _gpu_hull3d_faces

    def vertices(c):
        r = hull_fn(c)
        return None if r is None else r[0]

    cand = _candidates(coords, group, vertices)
    r = hull_fn([c[cand] for c in coords])
    if r is None:
        raise _degenerate()
    v, off, idx = r
    return cand[v.to(torch.long)], off.to(torch.long), cand[idx.to(torch.long)]


def sharded_hull3d_numpy(coords: Sequence[np.ndarray], hull_fn: Callable, group=None):
    """sharded_hull3d with numpy coordinates; hull_fn(coords) -> (vertices,
    list of faces) as numpy arrays, or None when the points do not span 3D
    (tests on CPU ranks).  Returns (vertices, list of faces) in global
    indices."""
    tc = [torch.from_numpy(np.ascontiguousarray(c)) for c in coords]

    def fn(parts):
        r = hull_fn([p.numpy() for p in parts])
        if r is None:
            return None
        v, faces = r
        off = np.zeros(len(faces) + 1, np.int64)
        off[1:] = np.cumsum([len(f) for f in faces])
        idx = np.concatenate([np.asarray(f, np.int64) for f in faces]) if faces else \
            np.zeros(0, np.int64)
        return (torch.from_numpy(np.asarray(v, np.int64)), torch.from_numpy(off),
                torch.from_numpy(idx))

    v, off, idx = sharded_hull3d(tc, group=group, hull_fn=fn)
    v, off, idx = v.numpy(), off.numpy(), idx.numpy()
    return v, [idx[off[i]:off[i + 1]] for i in range(len(off) - 1)]


def sharded_hull_numpy(coords: Sequence[np.ndarray], hull_fn: Callable, group=None):
    """The same with numpy coordinates and a numpy hull function (tests on
    CPU ranks)."""
    tc = [torch.from_numpy(np.ascontiguousarray(c)) for c in coords]

    def fn(parts):
        r = hull_fn([p.numpy() for p in parts])
        return None if r is None else torch.from_numpy(np.asarray(r, np.int64))

    final, cand = sharded_hull(tc, group=group, hull_fn=fn)
    return final.numpy(), cand.numpy()


class ShardedHull2D:
    """2D hulls of k clouds (k <= 8), each split into contiguous shards over
    the ranks of `group`, with every device step in the library's kernels:

      1. this rank's shards of all clouds in one persistent launch
         (qh_hull2d_multi_async);
      2. its rank block: shard-hull indices made global, with their
         coordinates (qh_shard_local);
      3. one all-gather of the fixed-size rank blocks (NCCL between GPUs);
      4. the candidate clouds, rank blocks in rank order (qh_shard_pack);
      5. their hulls in one persistent launch, then candidate-local indices
         mapped to global ones (qh_shard_remap).

    A rank holds only its shards.  No step synchronises with the host; the
    counts and statuses are read by results().  `shards[c]` is this rank's
    [2, hi - lo] float32 CUDA tensor (or (x, y) pair) of cloud c and
    `lo[c]` its first global index.  `cap` bounds a shard hull's size (a
    larger one is reported by results() as QH_ERR_CAPACITY).  For a
    one-process run of several ranks' blocks (tests), call local_block() for
    each and merge() on the stacked blocks."""

    def __init__(self, shards, lo, world: int, rank: int, cap: int = 16384, group=None):
        from . import Workspace, RESULT_BYTES, make_opts, _native
        self._n = _native
        self.k, self.world, self.rank, self.cap, self.group = len(shards), world, rank, cap, group
        if not 1 <= self.k <= 8:
            raise ValueError("1..8 clouds")
        self.shards = [(s[0], s[1]) if isinstance(s, torch.Tensor) else tuple(s) for s in shards]
        dev = self.shards[0][0].device
        self.lo = [int(v) for v in lo]
        self.opts = make_opts("f32", "persistent")
        self.words = int(_native.lib().qh_shard_block_words(2, cap))
        self.m = world * cap
        i32 = torch.int32
        self.local_out = [torch.empty(max(int(x.numel()), 1), dtype=i32, device=dev)
                          for x, _ in self.shards]
        self.local_res = torch.zeros(self.k * RESULT_BYTES, dtype=torch.uint8, device=dev)
        self.local_ws = Workspace(dev)
        self.block = torch.zeros(self.k * self.words, dtype=i32, device=dev)
        self.gathered = torch.zeros(world * self.k * self.words, dtype=i32, device=dev)
        self.ccoord = torch.zeros(2 * self.k * self.m, dtype=torch.float32, device=dev)
        self.cidx = torch.zeros(self.k * self.m, dtype=i32, device=dev)
        self.bad = torch.zeros(self.k, dtype=i32, device=dev)
        self.final_out = [torch.empty(self.m, dtype=i32, device=dev) for _ in range(self.k)]
        self.final_res = torch.zeros(self.k * RESULT_BYTES, dtype=torch.uint8, device=dev)
        self.final_ws = Workspace(dev)
        cc = self.ccoord.view(2, self.k, self.m)
        self.cands = [(cc[0, c], cc[1, c]) for c in range(self.k)]

    def _ptrs(self, ts):
        return (ctypes.c_void_p * len(ts))(*[t.data_ptr() for t in ts])

    def local_block(self, shards=None, lo=None, block=None, stream=None):
        """Steps 1-2 for the given shards (default: this rank's) into `block`."""
        from . import hull2d_multi_async, QHError, _stream_handle
        shards = self.shards if shards is None else shards
        lo = self.lo if lo is None else lo
        block = self.block if block is None else block
        hull2d_multi_async(list(shards), self.local_out, self.local_res, self.local_ws, self.opts,
                           stream)
        coords = []
        for x, y in shards:
            coords += [x, y]
        los = (ctypes.c_int64 * self.k)(*lo)
        st = self._n.lib().qh_shard_local(self.k, 2, self._ptrs(self.local_out),
                                          self.local_res.data_ptr(), los, self._ptrs(coords), 1,
                                          self.cap, block.data_ptr(), _stream_handle(stream))
        if st != 0:
            raise QHError(st, "qh_shard_local")
        return block

    def exchange(self):
        """Step 3: all-gather of the rank blocks."""
        if self.world > 1:
            dist.all_gather_into_tensor(self.gathered, self.block, group=self.group)
        else:
            self.gathered.copy_(self.block)

    def merge(self, gathered=None, stream=None):
        """Steps 4-5 on the gathered blocks ([world][k][words] int32)."""
        from . import hull2d_multi_async, QHError, _stream_handle
        g = self.gathered if gathered is None else gathered
        self.bad.zero_()
        st = self._n.lib().qh_shard_pack(self.k, 2, g.data_ptr(), self.world, self.cap,
                                         self.ccoord.data_ptr(), self.cidx.data_ptr(),
                                         self.bad.data_ptr(), _stream_handle(stream))
        if st != 0:
            raise QHError(st, "qh_shard_pack")
        hull2d_multi_async(self.cands, self.final_out, self.final_res, self.final_ws, self.opts,
                           stream)
        st = self._n.lib().qh_shard_remap(self.k, self._ptrs(self.final_out),
                                          self.final_res.data_ptr(), self.cidx.data_ptr(),
                                          self.m, _stream_handle(stream))
        if st != 0:
            raise QHError(st, "qh_shard_remap")

    def step(self, stream=None):
        self.local_block(stream=stream)
        self.exchange()
        self.merge(stream=stream)

    def results(self):
        """(global hull indices per cloud, as int32 CUDA tensors; statuses).
        Synchronises."""
        from . import result_from_tensor, RESULT_BYTES
        torch.cuda.synchronize()
        res = [result_from_tensor(self.final_res[c * RESULT_BYTES:(c + 1) * RESULT_BYTES])
               for c in range(self.k)]
        bad = self.bad.cpu().tolist()
        st = [b or r.status for r, b in zip(res, bad)]
        return [self.final_out[c][: res[c].count] for c in range(self.k)], st
