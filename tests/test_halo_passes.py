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
    manager = mp.Manager()
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
