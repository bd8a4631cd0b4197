"""Splitting a list of independent images (tiles) across GPUs, one process per GPU.

Tiles unwrap independently, so a multi-GPU batched solve needs no data-path collective: each
rank takes a share of the tiles, unwraps its share as one batch, and writes its own results.
The shares are chosen by longest-processing-time-first greedy scheduling (LPT: sort by cost,
give each tile to the rank with the least load so far), whose makespan is within
4/3 - 1/(3m) of the optimum on m ranks (Graham, 1969).  Every rank computes the same split
from the same shape list, so no exchange is needed to agree on it.

The split is plain host arithmetic; `unwrap_sharded` runs one rank's share through the batched
solver.
"""
from __future__ import annotations

import heapq

# Calibration of the cost estimate (seconds on one GB300, split-bf16 folded form, 4096 x 4096):
# the preconditioner took 0.490 ms per CG iteration for 4096^2 * (4096 + 4096) / 2 padded
# multiply-add units, the stencil kernels 0.331 ms for 4096^2 pixels.
_DCT_S_PER_UNIT = 0.490e-3 / (4096.0 * 4096.0 * 8192.0 / 2.0)
_STENCIL_S_PER_PX = 0.331e-3 / (4096.0 * 4096.0)


def _rup(x, m):
    return (x + m - 1) // m * m


def tile_cost(H, W):
    """Estimated seconds of one CG iteration of an H x W image in a batched solve.

    The preconditioner is four dense products over the padded transform sizes: the folded
    form (both sides >= 256) pads each even/odd half to a multiple of 256 and does half the
    multiply-adds of the direct form, which pads each side to a multiple of 128.  The stencil
    kernels move a fixed number of bytes per pixel.  Only the ratios between tiles matter
    for the split; the iteration count of each tile is not known in advance and is taken equal.
    """
    H, W = int(H), int(W)
    if H < 1 or W < 1:
        raise ValueError(f"bad tile shape {H} x {W}")
    if H >= 256 and W >= 256:
        Hp, Wp = 2 * _rup((H + 1) // 2, 256), 2 * _rup((W + 1) // 2, 256)
        units = Hp * Wp * (Hp + Wp) / 2.0
    else:
        Hp, Wp = _rup(H, 128), _rup(W, 128)
        units = float(Hp * Wp * (Hp + Wp))
    return units * _DCT_S_PER_UNIT + H * W * _STENCIL_S_PER_PX


def lpt_partition(costs, n_parts):
    """Indices of `costs` split into `n_parts` lists by LPT greedy scheduling.

    Ties are broken deterministically: equal costs go in index order, and equal loads go to
    the lowest part number.  Each returned list is in ascending index order, so one part
    keeps the input order.
    """
    n_parts = int(n_parts)
    if n_parts < 1:
        raise ValueError("n_parts must be >= 1")
    costs = [float(c) for c in costs]
    if any(not c >= 0.0 for c in costs):
        raise ValueError("costs must be finite and >= 0")
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, p) for p in range(n_parts)]
    parts = [[] for _ in range(n_parts)]
    for i in order:
        load, p = heapq.heappop(heap)
        parts[p].append(i)
        heapq.heappush(heap, (load + costs[i], p))
    return [sorted(p) for p in parts]


def shard_tiles(shapes, rank, world):
    """The indices of `shapes` (a list of (H, W)) that rank `rank` of `world` unwraps."""
    rank, world = int(rank), int(world)
    if not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside a world of {world}")
    return lpt_partition([tile_cost(h, w) for h, w in shapes], world)[rank]


def part_loads(shapes, parts):
    """Estimated seconds per CG iteration of each part (sum of its tiles' costs)."""
    return [sum(tile_cost(*shapes[i]) for i in p) for p in parts]


def unwrap_sharded(Xs, cohs=None, rank=None, world=None, device="cuda", batch=None, **opts):
    """Unwraps this rank's share of the images `Xs` (2-D tensors; `cohs` their coherences or
    None) as one batched solve on `device`.

    `rank` and `world` default to those of the initialised torch.distributed process group
    (0 and 1 without one).  Only this rank's images are copied to `device` (as contiguous
    float32), so `Xs` may stay in host memory.  No collective is issued; a process that needs
    every result gathers them itself.  `batch` builds the solver from the share's shapes and
    `opts` (default: the package's Batch).  Returns (indices, Us, stats) for this rank's images,
    in ascending index order; all three are empty when the rank has no image.
    """
    import torch
    if rank is None or world is None:
        r, w = 0, 1
        if torch.distributed.is_available() and torch.distributed.is_initialized():
            r, w = torch.distributed.get_rank(), torch.distributed.get_world_size()
        rank = r if rank is None else rank
        world = w if world is None else world
    if cohs is not None and len(cohs) != len(Xs):
        raise ValueError("one coherence per image")
    shapes = []
    for X in Xs:
        if X.dim() != 2:
            raise ValueError("images must be 2-D")
        shapes.append((int(X.shape[0]), int(X.shape[1])))
    mine = shard_tiles(shapes, rank, world)
    if not mine:
        return [], [], []
    if batch is None:
        from . import Batch as batch

    def put(t):
        return t.to(device=device, dtype=torch.float32).contiguous()

    Xm = [put(Xs[i]) for i in mine]
    Cm = None if cohs is None else [put(cohs[i]) for i in mine]
    b = batch([shapes[i] for i in mine], **opts)
    try:
        Us, stats = b.unwrap(Xm, Cm)
    finally:
        b.close()
    return mine, Us, stats
