"""Seeded synthetic inputs: shapes, bounds, determinism and dose."""
import numpy as np

from paper_2205_06327_gb300 import synth


def test_workload_shapes_and_bounds():
    for cid, (N, M, S, H, W) in {1: (64, 64, 1, 192, 192), 2: (576, 128, 16, 384, 384)}.items():
        wl = synth.workload(cid)
        assert (wl.N, wl.M, wl.S, wl.H, wl.W) == (N, M, S, H, W)
        assert wl.pos.dtype == np.int32
        assert wl.pos.min() >= 0
        assert wl.pos[:, 0].max() <= H - M and wl.pos[:, 1].max() <= W - M
        assert wl.obj.shape == (S, H, W) and np.allclose(np.abs(wl.obj), 1.0)
        # raster order, x fastest
        assert np.all(np.diff(wl.pos[:, 1].reshape(-1, int(np.sqrt(N)))) > 0)


def test_perovskite_shape_small_raster():
    wl = synth.workload_perovskite(n_rows=3, n_cols=4)
    assert wl.obj.shape == (30, 640, 656) and wl.N == 12
    full = synth.raster_positions(126, 132, 4, 6, 2)
    assert len(full) == 16632
    assert full[:, 0].max() + 128 <= 640 and full[:, 1].max() + 128 <= 656


def test_determinism_and_probe_energy():
    a = synth.workload_multislice()
    b = synth.workload_multislice()
    assert np.array_equal(a.obj, b.obj) and np.array_equal(a.probe, b.probe)
    assert np.isclose(np.sum(np.abs(a.probe) ** 2), 1e4)
    c = synth.workload_single_slice()
    assert np.isclose(np.sum(np.abs(c.probe) ** 2), 1.0)


def test_poisson_counts_seeded():
    I = np.full((4, 8, 8), 3.0)
    p1 = synth.poisson_counts(I, 5)
    p2 = synth.poisson_counts(I, 5)
    assert p1.dtype == np.float32 and np.array_equal(p1, p2)
    assert abs(p1.mean() - 3.0) < 0.5


def test_multi_problem_shapes():
    shapes = synth.multi_problem_shapes()
    assert len(shapes) == 32
    for M, S, ny, nx, step in shapes:
        assert M in (64, 96, 128, 192, 256) and 1 <= S <= 24
        assert 256 <= ny * nx <= 4096 + ny
