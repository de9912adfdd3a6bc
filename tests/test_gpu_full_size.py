"""GPU parity at the full PbTiO3-shaped size, in the launch configuration the
benchmark times (16632 positions, 30 slices of 640 x 656, recompute mode with a
checkpoint every 5 slices, default workspace and chunking).

The whole evaluation is too large for the FP64 oracle, so the test compares
outputs the oracle can compute one by one:
- the object gradient on a sampled block of pixels in three slices: by Eq. 2
  and the locality of Sec. III it is the sum, over the positions whose windows
  cover the block, of their per-position gradients there (about 1300
  positions, evaluated by the oracle in a spawn process pool);
- the far fields of sampled positions from the forward model.
The gradient bar is the FP32 rounding floor of a 30-slice chain, measured on the
same positions by the single-precision error model (tests/helpers), as in the
other long-chain tests.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from paper_2205_06327_gb300 import synth
from tests.helpers import (TOL_FP32, c64, pool_init, pool_intensities, pool_region_grad, propagator, rel_l2,
                           start_object, to_dev)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SLICES = [0, 17, 29]
BLOCK = (300, 316, 200, 216)  # y0, y1, x0, x1


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda", 0)


@pytest.fixture(scope="module")
def pool():
    ctx = mp.get_context("spawn")
    p = ctx.Pool(max(1, min(os.cpu_count() or 1, 32)), initializer=pool_init,
                 initargs=("workload_perovskite", "perturbed", 3))
    yield p
    p.close()
    p.join()


def test_perovskite_full_size_sampled(dev, pool):
    from paper_2205_06327_gb300 import api
    wl = synth.workload_perovskite()
    assert wl.N == 16632
    # Poisson data from the oracle's intensities at the true object
    chunks = np.array_split(np.arange(wl.N), 4 * (os.cpu_count() or 1))
    I = np.concatenate(pool.map(pool_intensities, chunks))
    I = synth.poisson_counts(I, 1003)
    start = start_object(wl, "perturbed", 3)

    g = api.Geometry(wl.M, wl.S, wl.H, wl.W, wl.N, wl.lambda_A, wl.dz_A, wl.pixel_A)
    plan = api.Plan(g, dev, async_check=True, ckpt_every=5)
    pos_d = to_dev(wl.pos, torch.int32, dev)
    probe_d = to_dev(wl.probe, torch.complex64, dev)
    obj_d = to_dev(start, torch.complex64, dev)
    I_d = to_dev(I, torch.float32, dev)
    _, gO, _ = plan.loss_grad(pos_d, probe_d, obj_d, I_d)
    y0, y1, x0, x1 = BLOCK
    go = gO[SLICES, y0:y1, x0:x1].cpu().numpy()
    psi, _ = plan.forward(pos_d, probe_d, obj_d, want_psi=True)
    sample = np.linspace(0, wl.N - 1, 8).astype(int)
    psi_s = psi[torch.from_numpy(sample).to(dev)].cpu().numpy()
    plan.close()
    del I_d, psi, gO

    M = wl.M
    cover = [i for i, (y, x) in enumerate(wl.pos) if y < y1 and y + M > y0 and x < x1 and x + M > x0]
    assert len(cover) > 1000
    parts = pool.map(pool_region_grad, [(i, I[i], SLICES, y0, y1, x0, x1) for i in cover], chunksize=8)
    ref = np.zeros((len(SLICES), y1 - y0, x1 - x0), np.complex128)
    f32 = np.zeros_like(ref)
    for p in parts:  # fixed order
        ref += p[0]
        f32 += p[1]
    e = rel_l2(go, ref)
    bar = max(TOL_FP32, 1.5 * rel_l2(f32, ref))
    print(f"gO on {len(SLICES)} x 16 x 16 pixels from {len(cover)} positions: {e:.2e} (bar {bar:.1e})")
    assert e <= bar

    Psi = orc.forward(c64(wl.probe), c64(start), wl.pos[sample], propagator(wl))
    ef = rel_l2(psi_s, Psi)
    print(f"far fields of {len(sample)} sampled positions: {ef:.2e}")
    assert ef <= TOL_FP32
