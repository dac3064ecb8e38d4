"""One hull over several ranks (one GPU each).

The hull of a union is the hull of the union of the parts' hulls, so a
cloud split into contiguous shards needs one exchange: every rank hulls its
shard, the shard hulls' vertices (global indices and coordinates) are
all-gathered, and the hull of the gathered vertices is the answer (computed
on every rank).  Only the shard hulls travel: h_g points per rank, small
next to n / G except for points on a circle or sphere.

`hull_fn` computes a hull on one rank's data and returns local indices; by
default it is the library's GPU hull.  The collective is torch.distributed
(NCCL between GPUs; the tests run it with gloo on CPU ranks).
"""
from __future__ import annotations

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


def _gpu_hull(coords: Sequence[torch.Tensor]):
    from . import hull2d, hull3d
    if len(coords) == 2:
        return hull2d(coords[0], coords[1]).long()
    v, _, _ = hull3d(coords[0], coords[1], coords[2])
    return v.long()


def sharded_hull(coords: Sequence[torch.Tensor], group=None,
                 hull_fn: Optional[Callable] = None):
    """Hull of the whole cloud, whose coordinates every rank holds (1-D
    tensors of the same length n).  Each rank hulls its shard; returns the
    global indices of the final hull as hull_fn orders them (2D: CCW from the
    lexicographic min; 3D: increasing vertex indices) and the gathered
    candidate indices.  In 3D the faces of the final hull are those of
    hull_fn on the gathered points, re-indexed by the caller if needed."""
    hull_fn = hull_fn or _gpu_hull
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    n = int(coords[0].numel())
    lo, hi = shard_range(n, rank, world)
    local = hull_fn([c[lo:hi] for c in coords]) if hi > lo else \
        torch.zeros(0, dtype=torch.long, device=coords[0].device)
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
    # candidates in increasing global index, so that duplicate locations keep
    # their lowest index as in the one-rank hull
    cand, _ = torch.sort(cand)
    sub = hull_fn([c[cand] for c in coords])
    return cand[sub.to(torch.long)], cand


def sharded_hull_numpy(coords: Sequence[np.ndarray], hull_fn: Callable, group=None):
    """The same with numpy coordinates and a numpy hull function (tests on
    CPU ranks)."""
    tc = [torch.from_numpy(np.ascontiguousarray(c)) for c in coords]

    def fn(parts):
        return torch.from_numpy(np.asarray(hull_fn([p.numpy() for p in parts]), np.int64))

    final, cand = sharded_hull(tc, group=group, hull_fn=fn)
    return final.numpy(), cand.numpy()
