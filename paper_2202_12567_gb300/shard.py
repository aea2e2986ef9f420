"""One frame over several processes (one GPU each), sharded by slices.

Slices are independent after setup (Sec. 3: every slice is sampled and completed on
its own), so a frame shards with no exchange on the data path: the slices are split
by longest-processing-time on their estimated cost, every rank renders its slices,
and the pixel blocks are gathered once at the end.  The functions here are the
host side of that split; they run on any torch.distributed backend (gloo on CPU,
NCCL between GPUs).
"""
from __future__ import annotations

import copy
import heapq

import numpy as np
import torch
import torch.distributed as dist


def slice_costs(slice_off, ncol=None, C: int | None = None) -> np.ndarray:
    """Estimated cost of each slice: m'_s n'_s entries to sample and complete (the
    global cut size C stands in for n'_s before pass 1)."""
    sizes = np.diff(np.asarray(slice_off, dtype=np.int64))
    n = np.asarray(ncol, dtype=np.int64) if ncol is not None else np.full(sizes.size, int(C or 1))
    return sizes * np.maximum(n, 1)


def lpt_partition(costs, world: int):
    """Slices per rank: largest cost first onto the least-loaded rank (ties: lower
    slice index, lower rank).  Returns sorted slice lists."""
    order = sorted(range(len(costs)), key=lambda s: (-int(costs[s]), s))
    heap = [(0, r) for r in range(world)]
    out = [[] for _ in range(world)]
    for s in order:
        load, r = heapq.heappop(heap)
        out[r].append(s)
        heapq.heappush(heap, (load + int(costs[s]), r))
    return [sorted(x) for x in out]


def rows_of(slice_off, slices) -> np.ndarray:
    """Slice-ordered rows of the given slices."""
    off = np.asarray(slice_off, dtype=np.int64)
    if len(slices) == 0:
        return np.zeros(0, dtype=np.int64)
    return np.concatenate([np.arange(off[s], off[s + 1]) for s in slices])


def gather_image(pixels: torch.Tensor, values: torch.Tensor, m: int, dst: int = 0, group=None):
    """Every rank holds values [k, ...] at pixel indices [k]; rank `dst` returns the
    full image [m, ...] (other ranks None), e.g. [m] or [m, 3] for colour.  Blocks of
    different sizes are padded to the largest."""
    world = dist.get_world_size(group)
    tail = tuple(values.shape[1:])
    n = torch.tensor([pixels.numel()], dtype=torch.int64)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    cap = int(max(int(x.item()) for x in sizes))
    pad_p = torch.full((cap,), -1, dtype=torch.int64)
    pad_v = torch.zeros((cap,) + tail, dtype=values.dtype)
    pad_p[:pixels.numel()] = pixels.to(torch.int64).cpu()
    pad_v[:pixels.numel()] = values.cpu()
    all_p = [torch.empty(cap, dtype=torch.int64) for _ in range(world)]
    all_v = [torch.empty((cap,) + tail, dtype=values.dtype) for _ in range(world)]
    dist.all_gather(all_p, pad_p, group=group)
    dist.all_gather(all_v, pad_v, group=group)
    if dist.get_rank(group) != dst:
        return None
    img = torch.zeros((m,) + tail, dtype=values.dtype)
    seen = torch.zeros(m, dtype=torch.bool)
    for p, v, k in zip(all_p, all_v, sizes):
        k = int(k.item())
        p, v = p[:k], v[:k]
        if bool(seen[p].any()):
            raise RuntimeError("a pixel was rendered by two ranks")
        img[p] = v
        seen[p] = True
    if not bool(seen.all()):
        raise RuntimeError("pixels missing from the gathered image")
    return img


def max_over_ranks(x: float, group=None, device=None) -> float:
    """The largest value over the ranks (the frame time of a sharded run)."""
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def shard_renderer(R, slices):
    """A renderer for the given slices of the frame that the set-up renderer R holds:
    their points (slice order kept), the same VPLs, tree, cut and forest, and each
    slice's index in the whole frame (lt_frame.slice_id), so every random draw is the
    one the whole frame makes and the shard's pixels equal the whole frame's.  Its
    image is full-size; only the shard's pixels (`pixels`) are written.  None when
    `slices` is empty."""
    from . import lt
    if len(slices) == 0:
        return None
    slices = [int(s) for s in slices]
    off = R.slice_off.cpu().numpy().astype(np.int64)
    rows = torch.from_numpy(rows_of(off, slices)).to(R.dev)
    sizes = [int(off[s + 1] - off[s]) for s in slices]
    sub = copy.copy(R)
    sub.pts_s = R.pts_s[:, rows].contiguous()
    sub.row_perm = R.row_perm[rows].contiguous()
    sub.slice_off = torch.tensor(np.concatenate([[0], np.cumsum(sizes)]), dtype=torch.int32, device=R.dev)
    sub.slice_id = torch.tensor(slices, dtype=torch.int32, device=R.dev)
    f = R.frame
    sub.frame = lt.Frame(sub.pts_s, R.vpls, sub.slice_off, R.tree, f.cut, f.forest, f.level_off, f.level_nodes, f.H,
                         slice_id=sub.slice_id)
    sub.smp = lt.Samples(sub.frame, R.cfg["rate"], R.cfg["rate1"])
    sub.uv = lt.Factors(sub.frame, R.cfg["rank"], per_slice=int(R.cfg.get("rank_cols", 0)) > 0)
    sub.img = torch.zeros(R.frame.m, dtype=torch.float32, device=R.dev)
    sub.graph = None
    sub.pixels = sub.row_perm.to(torch.int64)
    return sub
