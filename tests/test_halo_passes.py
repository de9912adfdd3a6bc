"""The paper's image-gradient decomposition across ranks (Sec. III-IV), on CPU.

R x C gloo ranks each accumulate the gradients of the positions whose window
centre lies in their tile (FP64 oracle per-position gradients, Eq. 2), run
the vertical/horizontal forward (add) and backward (replace) passes, and must
then hold the global gradient restricted to their extended tile; the stitched
cores must equal the global gradient.  Windows wider than a tile make extended
tiles overlap non-adjacent tiles (Fig. 4 c-d), which the passes carry through
the tile in between.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.multiprocessing as mp

from oracle import ptycho_oracle as orc
from paper_2205_06327_gb300 import synth


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(M=16, S=2, ny=8, nx=8, step=2, seed=123):
    wl = synth.workload_random(M, S, ny, nx, step, seed=seed, amp_jitter=0.1)
    h = orc.fresnel_propagator(wl.M, wl.lambda_A, wl.dz_A, wl.pixel_A)
    I = orc.intensities(wl.probe, wl.obj, wl.pos, h) * 1.3
    obj = wl.obj * np.exp(0.1j * synth.rng(seed).standard_normal(wl.obj.shape))
    return wl, obj, I, h


def _worker(rank, world, R, C, port, out):
    import torch.distributed as dist

    from paper_2205_06327_gb300 import halo_passes as hp
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl, obj, I, h = _problem()
    grid = hp.tile_grid(wl.H, wl.W, R, C, wl.pos, wl.M)
    me = grid[rank // C][rank % C]
    ys = np.array([grid[r][0].core.y0 for r in range(R)] + [wl.H])
    xs = np.array([grid[0][c].core.x0 for c in range(C)] + [wl.W])
    owner = hp.assign_positions(wl.pos, wl.M, ys, xs)
    e = me.ext
    buf = torch.zeros((wl.S, e.y1 - e.y0, e.x1 - e.x0), dtype=torch.complex128)
    for i in np.nonzero(owner == rank)[0]:
        _, gOi, _ = orc.position_loss_grad(wl.probe, obj, wl.pos[i], I[i], h)
        y, x = wl.pos[i] - np.array([e.y0, e.x0])
        buf[:, y:y + wl.M, x:x + wl.M] += torch.from_numpy(gOi)
    hp.exchange(buf, grid, me)
    _, gO, _ = orc.loss_grad(wl.probe, obj, wl.pos, I, h)
    ref = gO[:, e.y0:e.y1, e.x0:e.x1]
    out[rank] = (float(np.abs(buf.numpy() - ref).max()), float(np.abs(ref).max()),
                 int((owner == rank).sum()), (e.y0, e.y1, e.x0, e.x1), (me.core.y0, me.core.y1, me.core.x0, me.core.x1))
    dist.destroy_process_group()


@pytest.mark.parametrize("R,C", [(2, 2), (3, 3), (1, 3)])
def test_passes_give_the_global_gradient_on_every_extended_tile(R, C):
    world = R * C
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, R, C, _free_port(), out), nprocs=world, join=True)
    wl, _, _, _ = _problem()
    assert sum(out[k][2] for k in range(world)) == wl.N        # every position owned once
    for k in range(world):
        err, scale, _, ext, core = out[k]
        assert err <= 1e-12 * scale, (k, err, scale)
    if (R, C) == (3, 3):  # extended tiles of non-adjacent tiles overlap (Fig. 4 c-d)
        exts = [out[k][3] for k in range(world)]
        assert exts[0][3] > exts[2][2] and exts[0][1] > exts[6][0]


def test_stitching_the_cores_recovers_the_image():
    from paper_2205_06327_gb300 import halo_passes as hp
    wl, obj, I, h = _problem()
    grid = hp.tile_grid(wl.H, wl.W, 2, 3, wl.pos, wl.M)
    _, gO, _ = orc.loss_grad(wl.probe, obj, wl.pos, I, h)
    pieces = []
    for row in grid:
        for t in row:
            e = t.ext
            pieces.append((t, torch.from_numpy(gO[:, e.y0:e.y1, e.x0:e.x1].copy())))
    st = hp.stitch(pieces, gO.shape)
    assert np.array_equal(st.numpy(), gO)


# ------------------------------------------------ Algorithm 1: pipelined schedule with period T

ALPHA = 2e-3


def _grad_fn(wl, I, h, e):
    """Location i's object gradient on the extended tile e (oracle, FP64)."""
    def f(i, tile):
        y, x = int(wl.pos[i][0]) - e.y0, int(wl.pos[i][1]) - e.x0
        _, gOi, _ = orc.position_loss_grad(wl.probe, tile.numpy(), np.array([y, x]), I[i], h)
        g = torch.zeros_like(tile)
        g[:, y:y + wl.M, x:x + wl.M] = torch.from_numpy(gOi)
        return g
    return f


def _owned(wl, grid, R, C):
    from paper_2205_06327_gb300 import halo_passes as hp
    ys = np.array([grid[r][0].core.y0 for r in range(R)] + [wl.H])
    xs = np.array([grid[0][c].core.x0 for c in range(C)] + [wl.W])
    return hp.assign_positions(wl.pos, wl.M, ys, xs)


def _appp_worker(rank, world, R, C, T, epochs, port, out):
    import torch.distributed as dist

    from paper_2205_06327_gb300 import halo_passes as hp
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    wl, obj, I, h = _problem()
    grid = hp.tile_grid(wl.H, wl.W, R, C, wl.pos, wl.M)
    me = grid[rank // C][rank % C]
    e = me.ext
    mine = np.nonzero(_owned(wl, grid, R, C) == rank)[0]
    tile = torch.from_numpy(obj[:, e.y0:e.y1, e.x0:e.x1].copy())
    acc = torch.zeros_like(tile)
    for _ in range(epochs):
        hp.appp_epoch(tile, acc, grid, me, mine, _grad_fn(wl, I, h, e), ALPHA, T)
    out[rank] = tile.numpy()
    dist.destroy_process_group()


def _appp_reference(R, C, T, epochs):
    """The same schedule in one process: every tile's own loop, and at each
    common exchange point the global sum of all buffers, restricted to each
    extended tile (what the four passes deliver, tested above)."""
    from paper_2205_06327_gb300 import halo_passes as hp
    wl, obj, I, h = _problem()
    grid = hp.tile_grid(wl.H, wl.W, R, C, wl.pos, wl.M)
    owner = _owned(wl, grid, R, C)
    tiles = [t for row in grid for t in row]
    mine = [np.nonzero(owner == k)[0] for k in range(len(tiles))]
    V = [torch.from_numpy(obj[:, t.ext.y0:t.ext.y1, t.ext.x0:t.ext.x1].copy()) for t in tiles]
    acc = [torch.zeros_like(v) for v in V]
    n_max = max(len(m) for m in mine)
    for _ in range(epochs):
        for i in range(1, n_max + 1):
            for k, t in enumerate(tiles):
                if i <= len(mine[k]):
                    g = _grad_fn(wl, I, h, t.ext)(int(mine[k][i - 1]), V[k])
                    acc[k] += g
                    V[k] -= ALPHA * g
            if i % T == 0:
                G = torch.zeros(obj.shape, dtype=torch.complex128)
                for k, t in enumerate(tiles):
                    G[:, t.ext.y0:t.ext.y1, t.ext.x0:t.ext.x1] += acc[k]
                for k, t in enumerate(tiles):
                    V[k] -= ALPHA * G[:, t.ext.y0:t.ext.y1, t.ext.x0:t.ext.x1]
                    acc[k].zero_()
    return [v.numpy() for v in V]


@pytest.mark.parametrize("R,C,T,epochs", [(2, 2, 3, 2), (2, 2, 1000, 1), (1, 3, 5, 1)])
def test_appp_schedule_matches_the_reconciled_reference(R, C, T, epochs):
    """Algorithm 1 on gloo ranks: per-location updates of each extended tile, the
    buffers reconciled by the passes every T locations (T = 1000: once, after
    the largest rank's last location), then the second update."""
    world = R * C
    manager = mp.get_context("spawn").Manager()
    out = manager.dict()
    mp.spawn(_appp_worker, args=(world, R, C, T, epochs, _free_port(), out), nprocs=world, join=True)
    ref = _appp_reference(R, C, T, epochs)
    for k in range(world):
        scale = np.abs(ref[k]).max()
        assert np.abs(out[k] - ref[k]).max() <= 1e-12 * scale, k


def test_appp_single_tile_period_one_is_sgd_with_twice_the_step():
    """One tile, T = 1: the pass has no neighbour, so each location's gradient
    is applied twice, i.e. plain per-location descent with step 2 alpha."""
    import torch.distributed as dist

    from paper_2205_06327_gb300 import halo_passes as hp
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(_free_port()))
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        wl, obj, I, h = _problem()
        grid = hp.tile_grid(wl.H, wl.W, 1, 1, wl.pos, wl.M)
        me = grid[0][0]
        e = me.ext
        f = _grad_fn(wl, I, h, e)
        tile = torch.from_numpy(obj[:, e.y0:e.y1, e.x0:e.x1].copy())
        order = np.arange(wl.N)
        hp.appp_epoch(tile, torch.zeros_like(tile), grid, me, order, f, ALPHA, 1)
        ref = torch.from_numpy(obj[:, e.y0:e.y1, e.x0:e.x1].copy())
        for i in order:
            ref -= 2 * ALPHA * f(int(i), ref)
        assert np.abs(tile.numpy() - ref.numpy()).max() <= 1e-12 * np.abs(ref.numpy()).max()
    finally:
        dist.destroy_process_group()
