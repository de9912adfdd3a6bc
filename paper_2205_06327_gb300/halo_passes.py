"""Image-gradient decomposition across ranks: tiles, halos and the four passes.

The paper tessellates the image gradient into an R x C grid of tiles, one per
GPU (Sec. III).  Each tile is extended by a halo so that it covers the probe
windows of the positions assigned to it; its accumulation buffer holds the
sum of those positions' gradients (Eq. 2 restricted to the tile's
positions).  Overlapping parts of neighbouring buffers are then reconciled by
passes between neighbours (Sec. IV, Fig. 5): a vertical forward pass adds each
tile's overlap into the tile below, a vertical backward pass replaces each
tile's overlap with the (now complete) values of the tile below, and the same
two passes run horizontally.  Because extended tiles are products of a row
interval and a column interval, the vertical passes give column sums and the
horizontal passes complete them: afterwards every buffer equals the global
gradient restricted to its extended tile.

On one GPU the library sums the gradient with the owner-computes tiled
accumulation instead; this module runs the decomposition over any
torch.distributed process group (gloo ranks on CPU in the tests), with
non-blocking point-to-point messages as in the paper's asynchronous passes.
:func:`appp_epoch` runs the paper's pipelined schedule (Algorithm 1) on top of them:
per-location updates of each extended tile, with the accumulated gradients
reconciled every T locations.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch
import torch.distributed as dist


@dataclass(frozen=True)
class Rect:
    y0: int
    y1: int  # exclusive
    x0: int
    x1: int  # exclusive

    def intersect(self, o: "Rect") -> "Rect | None":
        y0, y1, x0, x1 = max(self.y0, o.y0), min(self.y1, o.y1), max(self.x0, o.x0), min(self.x1, o.x1)
        return Rect(y0, y1, x0, x1) if y0 < y1 and x0 < x1 else None


@dataclass(frozen=True)
class Tile:
    r: int
    c: int
    core: Rect      # the tile itself
    ext: Rect       # tile plus halo (clipped to the image)


def tile_grid(H: int, W: int, R: int, C: int, pos: np.ndarray, M: int) -> list[list[Tile]]:
    """R x C tiles of the H x W image; positions go to the tile containing the
    centre of their window; each extended tile is the bounding box of its core
    and of its positions' windows (the halo the paper sizes from the probe
    radius)."""
    ys = np.linspace(0, H, R + 1).round().astype(int)
    xs = np.linspace(0, W, C + 1).round().astype(int)
    owner = assign_positions(pos, M, ys, xs)
    grid = []
    for r in range(R):
        row = []
        for c in range(C):
            core = Rect(int(ys[r]), int(ys[r + 1]), int(xs[c]), int(xs[c + 1]))
            y0, y1, x0, x1 = core.y0, core.y1, core.x0, core.x1
            mine = pos[owner == r * C + c]
            if len(mine):
                y0 = min(y0, int(mine[:, 0].min()))
                y1 = max(y1, int(mine[:, 0].max()) + M)
                x0 = min(x0, int(mine[:, 1].min()))
                x1 = max(x1, int(mine[:, 1].max()) + M)
            row.append(Tile(r, c, core, Rect(max(0, y0), min(H, y1), max(0, x0), min(W, x1))))
        grid.append(row)
    # halos wide enough that every extended tile contains its neighbours' overlaps
    # along rows and columns: use the row-wise / column-wise envelope
    R_, C_ = len(grid), len(grid[0])
    yint = [(min(grid[r][c].ext.y0 for c in range(C_)), max(grid[r][c].ext.y1 for c in range(C_))) for r in range(R_)]
    xint = [(min(grid[r][c].ext.x0 for r in range(R_)), max(grid[r][c].ext.x1 for r in range(R_))) for c in range(C_)]
    return [[Tile(r, c, grid[r][c].core, Rect(yint[r][0], yint[r][1], xint[c][0], xint[c][1]))
             for c in range(C_)] for r in range(R_)]


def assign_positions(pos: np.ndarray, M: int, ys: np.ndarray, xs: np.ndarray) -> np.ndarray:
    """Flat tile index (r * C + c) owning each position (by window centre)."""
    cy = pos[:, 0] + M // 2
    cx = pos[:, 1] + M // 2
    r = np.clip(np.searchsorted(ys, cy, side="right") - 1, 0, len(ys) - 2)
    c = np.clip(np.searchsorted(xs, cx, side="right") - 1, 0, len(xs) - 2)
    return r * (len(xs) - 1) + c


def _real(t: torch.Tensor) -> torch.Tensor:
    """Messages travel as real tensors (complex values as (re, im) pairs)."""
    return torch.view_as_real(t) if t.is_complex() else t


def _view(buf: torch.Tensor, ext: Rect, reg: Rect) -> torch.Tensor:
    return buf[..., reg.y0 - ext.y0:reg.y1 - ext.y0, reg.x0 - ext.x0:reg.x1 - ext.x0]


def _pass(buf: torch.Tensor, grid, me: Tile, axis: int, forward: bool, rank_of, group=None) -> None:
    """One pass along an axis (0: vertical, 1: horizontal).  Forward: receive the
    previous neighbour's overlap and add it, then send ours to the next one.
    Backward: receive the next neighbour's overlap and replace ours with it,
    then send ours to the previous one."""
    R, C = len(grid), len(grid[0])
    n = R if axis == 0 else C
    k = me.r if axis == 0 else me.c

    def nb(j):
        return grid[j][me.c] if axis == 0 else grid[me.r][j]

    src = k - 1 if forward else k + 1
    dst = k + 1 if forward else k - 1
    if 0 <= src < n:
        other = nb(src)
        reg = me.ext.intersect(other.ext)
        if reg is not None:
            tmp = torch.empty_like(_view(buf, me.ext, reg)).contiguous()
            dist.irecv(_real(tmp), src=rank_of(other), group=group).wait()
            if forward:
                _view(buf, me.ext, reg).add_(tmp)
            else:
                _view(buf, me.ext, reg).copy_(tmp)
    if 0 <= dst < n:
        other = nb(dst)
        reg = me.ext.intersect(other.ext)
        if reg is not None:
            dist.isend(_real(_view(buf, me.ext, reg).contiguous()), dst=rank_of(other), group=group).wait()


def exchange(buf: torch.Tensor, grid, me: Tile, group=None) -> None:
    """The four passes of Sec. IV on this rank's accumulation buffer (in place):
    vertical forward, vertical backward, horizontal forward, horizontal backward.
    ``buf`` is [..., ext height, ext width] (e.g. [S, h, w] complex)."""
    C = len(grid[0])

    def rank_of(t: Tile) -> int:
        return t.r * C + t.c

    _pass(buf, grid, me, 0, True, rank_of, group)
    _pass(buf, grid, me, 0, False, rank_of, group)
    _pass(buf, grid, me, 1, True, rank_of, group)
    _pass(buf, grid, me, 1, False, rank_of, group)


def appp_epoch(buf_tile: torch.Tensor, acc: torch.Tensor, grid, me: Tile, my_pos: np.ndarray, grad_fn,
               alpha: float, T: int, group=None) -> None:
    """One pass over this rank's probe locations of the paper's asynchronous
    pipelined schedule (Algorithm 1), in place on its extended tile ``buf_tile``
    and its accumulated-gradient buffer ``acc`` (both [..., ext height, ext
    width]; ``acc`` carries over between passes).  For the i-th location
    (i = 1, 2, ...): its gradient g_i = grad_fn(index, buf_tile) (the tile's
    shape, zero outside the window), acc += g_i, tile -= alpha g_i; after
    every T-th location the four passes reconcile the buffers with the
    neighbours (:func:`exchange`), the tile takes a second step
    tile -= alpha acc, and acc is reset.  Ranks own different numbers of
    locations, so i follows a count common to all ranks (the largest rank's):
    a rank whose locations ran out still joins every exchange."""
    n = len(my_pos)
    cnt = torch.tensor([n], dtype=torch.int64)
    dist.all_reduce(cnt, op=dist.ReduceOp.MAX, group=group)
    n_max = int(cnt.item())
    for i in range(1, n_max + 1):
        if i <= n:
            g = grad_fn(int(my_pos[i - 1]), buf_tile)
            acc += g
            buf_tile -= alpha * g
        if i % T == 0:
            exchange(acc, grid, me, group)
            buf_tile -= alpha * acc
            acc.zero_()


def stitch(tiles_and_bufs, shape) -> torch.Tensor:
    """The final image from the cores of all tiles (halos dropped), as in Algorithm 1."""
    out = torch.zeros(shape, dtype=tiles_and_bufs[0][1].dtype)
    for t, b in tiles_and_bufs:
        out[..., t.core.y0:t.core.y1, t.core.x0:t.core.x1] = _view(b, t.ext, t.core)
    return out
