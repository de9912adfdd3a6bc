"""GPU parity: the CUDA path through the C-ABI against the FP64 oracle.

The oracle runs on the complex64 values the GPU receives.  Bar (FP32 path):
relative L2 error <= 1e-5 on the loss, and on both gradients wherever plain
FP32 arithmetic can reach it.  For long chains (16+ slices) the FFT rounding
of the forward chain, amplified by the amplitude residual, puts the gradient
error of any FP32 evaluation near 1e-5..3e-5; there the bar is 1.5x the error
of a SciPy single-precision evaluation of the same chain on the same inputs
(tests/helpers.fp32_chain_loss_grad), so the kernel must be as accurate as a
plain FP32 implementation (the loss bar likewise, where that model's loss
error exceeds 1e-5: the 100-slice chain of 1024^2 windows).  Where the
oracle's loss is 0 (noise-free data at the true object) the check is
absolute: F_gpu <= 1e-6 * sum(I).
"""
import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from paper_2205_06327_gb300 import synth
from tests.helpers import (TOL_FP32, c64, fp32_chain_loss_grad, measurements, propagator, rel_l2,
                           start_object, to_dev)

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda", 0)


def _plan(wl, dev, **kw):
    from paper_2205_06327_gb300 import api
    return api.Plan(api.Geometry(wl.M, wl.S, wl.H, wl.W, wl.N, wl.lambda_A, wl.dz_A, wl.pixel_A), dev, **kw)


def _run(wl, obj, I, dev, probe=None, **kw):
    plan = _plan(wl, dev, **kw)
    probe = wl.probe if probe is None else probe
    loss, gO, gP = plan.loss_grad(to_dev(wl.pos, torch.int32, dev), to_dev(probe, torch.complex64, dev),
                                  to_dev(obj, torch.complex64, dev), to_dev(I, torch.float32, dev))
    torch.cuda.synchronize()
    out = loss.item(), gO.cpu().numpy(), gP.cpu().numpy()
    plan.close()
    return out


def _check(wl, obj, I, dev, tol=TOL_FP32, fp32_floor=False, **kw):
    h = propagator(wl)
    L, gO, gP = orc.loss_grad(c64(wl.probe), c64(obj), wl.pos, I.astype(np.float64), h)
    l, go, gp = _run(wl, obj, I, dev, **kw)
    el = abs(l - L) / abs(L)
    eo, ep = rel_l2(go, gO), rel_l2(gp, gP)
    tol_l = tol_o = tol_p = tol
    if fp32_floor:
        lf, fo, fp = fp32_chain_loss_grad(wl.probe, obj, wl.pos, I, h)
        tol_l = max(tol, 1.5 * abs(lf - L) / abs(L))
        tol_o = max(tol, 1.5 * rel_l2(fo, gO))
        tol_p = max(tol, 1.5 * rel_l2(fp, gP))
    print(f"{wl.name}: loss {el:.2e} (bar {tol_l:.1e}) gO {eo:.2e} (bar {tol_o:.1e}) gP {ep:.2e} "
          f"(bar {tol_p:.1e})")
    assert el <= tol_l and eo <= tol_o and ep <= tol_p, (el, eo, ep)
    return l, go, gp


# --------------------------------------------------------------- workloads

def test_single_slice_workload_perturbed_start(dev):
    wl = synth.workload_single_slice()
    I = measurements(wl)
    _check(wl, start_object(wl, "perturbed", 1), I, dev)


def test_single_slice_workload_vacuum_start_loss(dev):
    """O = 1 with a band-limited probe: the far field is exactly zero outside the
    aperture, where the subgradient Psi/|Psi| is decided by rounding noise in any
    precision, so only the loss is comparable there."""
    wl = synth.workload_single_slice()
    I = measurements(wl)
    obj = start_object(wl, "vacuum")
    L = orc.loss(c64(wl.probe), obj, wl.pos, I.astype(np.float64), propagator(wl))
    l, _, _ = _run(wl, obj, I, dev)
    assert abs(l - L) <= TOL_FP32 * L


def test_zero_far_field_gives_zero_subgradient(dev):
    """P = 0: Psi = 0 exactly, F = sum(I) and the gradient is exactly 0 (|Psi| = 0 reading)."""
    wl = synth.workload_random(64, 3, 2, 2, 9, seed=21)
    I = (measurements(wl) + 0.5).astype(np.float32)
    l, go, gp = _run(wl, wl.obj, I, dev, probe=np.zeros_like(wl.probe))
    assert abs(l - float(I.astype(np.float64).sum())) <= 1e-6 * float(I.sum())
    assert not go.any() and not gp.any()


def test_single_slice_workload_at_truth_is_zero(dev):
    wl = synth.workload_single_slice()
    I = measurements(wl)
    l, go, gp = _run(wl, wl.obj, I, dev)
    assert l <= 1e-6 * float(I.sum())
    _, gO_ref, _ = orc.loss_grad(wl.probe, start_object(wl, "vacuum"), wl.pos, I.astype(np.float64), propagator(wl))
    assert np.linalg.norm(go) <= 1e-3 * np.linalg.norm(gO_ref)


def test_multislice_workload_full_size(dev):
    """All 576 positions, 16 slices of 384^2, Poisson data, perturbed start."""
    wl = synth.workload_multislice()
    I = measurements(wl, counts_seed=1002)
    _check(wl, start_object(wl, "perturbed", 2), I, dev, fp32_floor=True)


def test_multislice_workload_at_truth_with_noise(dev):
    wl = synth.workload_multislice()
    wl.pos = wl.pos[::7]
    I = measurements(wl, counts_seed=1002)
    _check(wl, wl.obj, I, dev, fp32_floor=True)


def test_multislice_eight_slices_strict(dev):
    """Half the slices of the 16-slice workload: plain FP32 meets 1e-5 on everything."""
    wl = synth.workload_multislice()
    wl.obj, wl.S = wl.obj[:8], 8
    wl.pos = wl.pos[::5]
    I = measurements(wl, counts_seed=1002)
    _check(wl, start_object(wl, "perturbed", 9), I, dev)


@pytest.mark.parametrize("M,S,ny,nx,step", [(64, 1, 3, 5, 7), (64, 5, 4, 3, 11), (128, 2, 2, 3, 20),
                                             (128, 7, 3, 3, 13)])
def test_random_problems_nonunimodular(dev, M, S, ny, nx, step):
    wl = synth.workload_random(M, S, ny, nx, step, seed=M + S, amp_jitter=0.2)
    I = (measurements(wl) * 1.2).astype(np.float32)
    _check(wl, start_object(wl, "perturbed", 5), I, dev)


def test_perovskite_subset(dev):
    """PbTiO3-shaped object (30 x 640x656) with a 6x7 block of the 4-px raster."""
    wl = synth.workload_perovskite(n_rows=6, n_cols=7)
    wl.pos = wl.pos + np.array([200, 240], np.int32)
    I = measurements(wl, counts_seed=1003)
    _check(wl, start_object(wl, "perturbed", 3), I, dev, fp32_floor=True)


# ------------------------------------------------------------------ forward

def test_forward_far_field_and_intensity(dev):
    from paper_2205_06327_gb300 import api
    wl = synth.workload_random(128, 3, 2, 2, 17, seed=3, amp_jitter=0.1)
    Psi = orc.forward(c64(wl.probe), c64(wl.obj), wl.pos, propagator(wl))
    plan = _plan(wl, dev)
    psi, inten = plan.forward(to_dev(wl.pos, torch.int32, dev), to_dev(wl.probe, torch.complex64, dev),
                              to_dev(wl.obj, torch.complex64, dev), want_psi=True, want_intensity=True)
    torch.cuda.synchronize()
    assert rel_l2(psi.cpu().numpy(), Psi) <= TOL_FP32
    assert rel_l2(inten.cpu().numpy(), np.abs(Psi) ** 2) <= TOL_FP32


# ------------------------------------------------------- structure and edges

def test_deterministic_bitwise(dev):
    wl = synth.workload_random(64, 4, 4, 4, 6, seed=11)
    I = (measurements(wl) * 0.8).astype(np.float32)
    obj = start_object(wl, "perturbed", 1)
    a = _run(wl, obj, I, dev)
    b = _run(wl, obj, I, dev)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_tiling_and_chunking_invariance(dev):
    """Eq. 2 / Sec. III: tile shape does not change the per-pixel summation order
    (bit-identical); chunking the positions only reassociates the sum."""
    wl = synth.workload_random(64, 3, 6, 5, 5, seed=12)
    I = (measurements(wl) * 1.1).astype(np.float32)
    obj = start_object(wl, "perturbed", 2)
    ref = _run(wl, obj, I, dev)
    tiled = _run(wl, obj, I, dev, tile=((wl.H + 7) // 8, (wl.W + 7) // 8))
    assert np.array_equal(ref[1], tiled[1])
    per_pos = (2 * wl.S - 1) * wl.M * wl.M * 8 + wl.M * wl.M * 8 + 8
    chunked = _run(wl, obj, I, dev, workspace_bytes=7 * per_pos)
    assert abs(chunked[0] - ref[0]) <= 1e-12 * abs(ref[0])
    assert rel_l2(chunked[1], ref[1]) <= 1e-6 and rel_l2(chunked[2], ref[2]) <= 1e-6


def test_window_at_object_corners(dev):
    wl = synth.workload_random(64, 2, 1, 1, 1, seed=13, amp_jitter=0.1)
    wl.pos = np.array([[0, 0], [wl.H - 64, wl.W - 64], [0, wl.W - 64], [wl.H - 64, 0]], np.int32)
    I = (measurements(wl) * 0.7).astype(np.float32)
    _check(wl, start_object(wl, "perturbed", 4), I, dev)


@pytest.mark.parametrize("M", [64, 128])
def test_repeated_and_unsorted_positions(dev, M):
    # The same window twice (both terms are summed, Eq. 2) and the positions in
    # a seeded random order (the library keeps the caller's order): the
    # oracle's sum over the same list.
    wl = synth.workload_random(M, 3, 3, 4, 9, seed=15 + M, amp_jitter=0.1)
    rep = np.concatenate([wl.pos, wl.pos[[1, 5, 5]]])
    wl.pos = rep[np.random.default_rng(16).permutation(len(rep))].astype(np.int32)
    I = (measurements(wl) * 0.9).astype(np.float32)
    _check(wl, start_object(wl, "perturbed", 6), I, dev)


def test_single_position(dev):
    wl = synth.workload_random(128, 4, 1, 1, 1, seed=17, amp_jitter=0.1)
    wl.pos = np.array([[wl.H - wl.M - 1, wl.W - wl.M]], np.int32)  # off the raster, at the right edge
    I = (measurements(wl) * 1.3).astype(np.float32)
    _check(wl, start_object(wl, "perturbed", 7), I, dev)


def test_zero_positions(dev):
    wl = synth.workload_random(64, 2, 1, 1, 1, seed=14)
    wl.pos = np.zeros((0, 2), np.int32)
    I = np.zeros((0, 64, 64), np.float32)
    l, go, gp = _run(wl, wl.obj, I, dev)
    assert l == 0.0 and not go.any() and not gp.any()


def test_errors_are_reported_not_faulted(dev):
    from paper_2205_06327_gb300 import api
    from paper_2205_06327_gb300._lib import PTYCHO_ERR_POSITION, PTYCHO_ERR_UNSUPPORTED, PtychoError
    wl = synth.workload_random(64, 2, 2, 2, 5, seed=15)
    I = measurements(wl)
    bad = wl.pos.copy()
    bad[1] = [wl.H - 63, 0]
    plan = _plan(wl, dev)
    args = (to_dev(bad, torch.int32, dev), to_dev(wl.probe, torch.complex64, dev),
            to_dev(wl.obj, torch.complex64, dev), to_dev(I, torch.float32, dev))
    with pytest.raises(PtychoError) as e:
        plan.loss_grad(*args)
    assert e.value.code == PTYCHO_ERR_POSITION
    # asynchronous check: the device skips the window and reports it afterwards
    aplan = _plan(wl, dev, async_check=True)
    aplan.loss_grad(*args)
    torch.cuda.synchronize()
    with pytest.raises(PtychoError) as e:
        aplan.status()
    assert e.value.code == PTYCHO_ERR_POSITION
    aplan.status()  # cleared
    with pytest.raises(PtychoError) as e:
        api.Plan(api.Geometry(100, 2, 200, 200, 4), dev)
    assert e.value.code == PTYCHO_ERR_UNSUPPORTED
    # the context is still usable
    _check(wl, wl.obj * 0.9, I, dev)


# --------------------------------------------------------- gradient checks

def test_gpu_gradient_matches_fp64_finite_differences(dev):
    """Directional derivatives of the FP64 loss (central differences) against
    Re<g_gpu, d> on the multislice workload (a block of 36 positions)."""
    wl = synth.workload_multislice()
    wl.pos = wl.pos.reshape(24, 24, 2)[8:14, 8:14].reshape(-1, 2).copy()
    I = measurements(wl, counts_seed=1002)
    obj = start_object(wl, "perturbed", 6)
    _, go, gp = _run(wl, obj, I, dev)
    h = propagator(wl)
    P0, O0 = c64(wl.probe), c64(obj)
    _, fo, fp = fp32_chain_loss_grad(wl.probe, obj, wl.pos, I, h)
    g = synth.rng(8)
    eps = 1e-6
    for _ in range(3):
        dO = g.standard_normal(obj.shape) + 1j * g.standard_normal(obj.shape)
        dP = g.standard_normal(wl.probe.shape) + 1j * g.standard_normal(wl.probe.shape)
        fd = (orc.loss(P0 + eps * dP, O0 + eps * dO, wl.pos, I.astype(np.float64), h)
              - orc.loss(P0 - eps * dP, O0 - eps * dO, wl.pos, I.astype(np.float64), h)) / (2 * eps)
        dd = lambda a, b: np.real(np.vdot(a.astype(np.complex128), dO) + np.vdot(b.astype(np.complex128), dP))
        an, model = dd(go, gp), dd(fo, fp)
        bar = max(1e-5, 1.5 * abs(model - fd) / abs(fd))
        print(f"directional derivative: gpu {abs(an - fd) / abs(fd):.2e}  fp32 model {abs(model - fd) / abs(fd):.2e}")
        assert abs(an - fd) <= bar * abs(fd), (an, fd, model)


def test_step_fixed_and_line_search(dev):
    from paper_2205_06327_gb300 import api
    wl = synth.workload_random(64, 3, 3, 3, 8, seed=16, amp_jitter=0.1)
    I = measurements(wl)
    obj = start_object(wl, "perturbed", 7)
    h = propagator(wl)
    plan = _plan(wl, dev)
    pos = to_dev(wl.pos, torch.int32, dev)
    Id = to_dev(I, torch.float32, dev)
    P = to_dev(wl.probe, torch.complex64, dev)
    O = to_dev(obj, torch.complex64, dev)
    a_o, a_p = 1e-3, 1e-5
    loss, t = plan.step(pos, P, O, Id, a_o, a_p)
    Pn, On, F0, _ = orc.step(wl.probe.astype(np.complex64).astype(np.complex128),
                             obj.astype(np.complex64).astype(np.complex128), wl.pos, I.astype(np.float64), h, a_o, a_p)
    assert t == 1.0 and abs(loss.item() - F0) <= 1e-5 * F0
    assert rel_l2(O.cpu().numpy(), On) <= 1e-6 and rel_l2(P.cpu().numpy(), Pn) <= 1e-6
    # Armijo with a deliberately large step backtracks and decreases the loss
    L0 = plan.loss_grad(pos, P, O, Id)[0].item()
    loss, t = plan.step(pos, P, O, Id, 50.0, 0.5, line_search=True)
    L1 = plan.loss_grad(pos, P, O, Id)[0].item()
    assert 0.0 < t < 1.0 and L1 < L0


def test_autograd_function(dev):
    from paper_2205_06327_gb300.autograd import ptycho_loss
    wl = synth.workload_random(64, 2, 2, 3, 9, seed=17)
    I = measurements(wl)
    obj0 = start_object(wl, "perturbed", 8)
    plan = _plan(wl, dev)
    O = to_dev(obj0, torch.complex64, dev).requires_grad_(True)
    P = to_dev(wl.probe, torch.complex64, dev).requires_grad_(True)
    L = ptycho_loss(O, P, plan, to_dev(wl.pos, torch.int32, dev), to_dev(I, torch.float32, dev))
    (2.0 * L).backward()
    Lr, gO, gP = orc.loss_grad(c64(wl.probe), c64(obj0), wl.pos, I.astype(np.float64), propagator(wl))
    assert abs(L.item() - Lr) <= 1e-5 * Lr
    assert rel_l2(O.grad.cpu().numpy(), 2 * gO) <= TOL_FP32
    assert rel_l2(P.grad.cpu().numpy(), 2 * gP) <= TOL_FP32


def test_potential_parameterisation(dev):
    """O = exp(i sigma V) and dF/dV = sigma Im(conj(O) dF/dO) against the oracle, and
    the autograd path over V against FP64 finite differences of the oracle loss."""
    from paper_2205_06327_gb300 import api
    from paper_2205_06327_gb300.autograd import ptycho_loss_potential
    wl = synth.workload_random(64, 3, 3, 3, 8, seed=31)
    sigma = 0.7
    V = (wl.potential / sigma).astype(np.float32)
    I = measurements(wl)
    Vd = to_dev(V, torch.float32, dev)
    O = api.potential_to_transmission(Vd, sigma)
    O_ref = np.exp(1j * sigma * V.astype(np.float64))
    assert rel_l2(O.cpu().numpy(), O_ref) <= 1e-6
    V0 = V + 0.05 * synth.rng(4).standard_normal(V.shape).astype(np.float32)
    plan = _plan(wl, dev)
    Vt = to_dev(V0, torch.float32, dev).requires_grad_(True)
    L = ptycho_loss_potential(Vt, to_dev(wl.probe, torch.complex64, dev), plan, to_dev(wl.pos, torch.int32, dev),
                              to_dev(I, torch.float32, dev), sigma)
    L.backward()
    O0 = np.exp(1j * sigma * V0.astype(np.float64))
    _, gO, _ = orc.loss_grad(c64(wl.probe), c64(O0), wl.pos, I.astype(np.float64), propagator(wl))
    gV_ref = orc.potential_grad(c64(O0), gO, sigma)
    assert rel_l2(Vt.grad.cpu().numpy(), gV_ref) <= TOL_FP32
    d = synth.rng(5).standard_normal(V.shape)
    e = 1e-4
    fd = (orc.loss(c64(wl.probe), np.exp(1j * sigma * (V0 + e * d)), wl.pos, I.astype(np.float64), propagator(wl))
          - orc.loss(c64(wl.probe), np.exp(1j * sigma * (V0 - e * d)), wl.pos, I.astype(np.float64),
                     propagator(wl))) / (2 * e)
    assert abs(float(np.sum(Vt.grad.cpu().numpy() * d)) - fd) <= 1e-4 * abs(fd)


@pytest.mark.parametrize("M,S,L", [(64, 7, 3), (128, 5, 2), (64, 4, 1), (128, 4, 3), (64, 6, 5)])
def test_recompute_mode_matches_store_all(dev, M, S, L):
    """Checkpoint every L slices + per-segment recomputation: the loss is
    bit-identical (same forward), the gradients agree with the store-all mode
    to FP32 reassociation and with the oracle at the usual bar, and the
    workspace per position shrinks."""
    wl = synth.workload_random(M, S, 3, 4, 9, seed=40 + M + S, amp_jitter=0.1)
    I = (measurements(wl) * 1.3).astype(np.float32)
    obj = start_object(wl, "perturbed", 6)
    ref = _run(wl, obj, I, dev)
    rc = _check(wl, obj, I, dev, ckpt_every=L)
    assert rc[0] == ref[0]
    assert rel_l2(rc[1], ref[1]) <= 2e-6 and rel_l2(rc[2], ref[2]) <= 2e-6
    p_all, p_rc = _plan(wl, dev), _plan(wl, dev, ckpt_every=L)
    K = -(-S // L)
    per = wl.M * wl.M * 8
    assert p_all.workspace_bytes // wl.N == (2 * S - 1) * per + per + 8
    assert p_rc.workspace_bytes // wl.N == (K + L - 1) * per + per + 8
    p_all.close()
    p_rc.close()


@pytest.mark.parametrize("M", [64, 128])
def test_recompute_workspace_does_not_hold_a_patch_per_slice(dev, M):
    """Per-position workspace in recompute mode is K - 2 checkpoints, one
    segment of L waves, the parked adjoint state and the probe gradient:
    for a fixed segment length it grows only by the checkpoints, never by a
    buffer per slice, and with the automatic choice (K = L = sqrt(S)) it is
    2 sqrt(S) buffers against 2S when every wave is kept."""
    from paper_2205_06327_gb300 import api
    per = M * M * 8
    for S, L in [(16, 4), (64, 4), (64, 8), (100, 10), (30, 5)]:
        g = api.Geometry(M, S, M + 8, M + 8, 4, 0.0251, 2.0, 0.1)
        p = api.Plan(g, dev, ckpt_every=L)
        K = -(-S // L)
        assert p.workspace_bytes // 4 == (K + L - 1) * per + per + 8, (S, L)
        p.close()
    for S in (16, 64):
        g = api.Geometry(M, S, M + 8, M + 8, 4, 0.0251, 2.0, 0.1)
        auto, full = api.Plan(g, dev, ckpt_every="auto"), api.Plan(g, dev)
        r = int(np.ceil(np.sqrt(S)))
        assert auto.workspace_bytes // 4 == 2 * r * per + 8
        assert full.workspace_bytes // 4 == 2 * S * per + 8
        auto.close()
        full.close()


@pytest.mark.parametrize("M", [64, 128, 96])
def test_recompute_mode_over_several_chunks(dev, M):
    """Recompute mode with a workspace that holds only a few positions: every
    chunk runs its K launches and per-segment accumulations (the later chunks
    adding to the gradient), and the results equal the store-all mode over one
    chunk to FP32 reassociation."""
    S, L = 5, 2
    wl = synth.workload_random(M, S, 3, 3, 11, seed=44 + M, amp_jitter=0.1)
    I = (measurements(wl) * 1.2).astype(np.float32)
    obj = start_object(wl, "perturbed", 9)
    K = -(-S // L)
    per = (K + L - 1 + (L + 1 if M not in (64, 128) else 0)) * M * M * 8 + M * M * 8 + 8
    small = _plan(wl, dev, ckpt_every=L, workspace_bytes=3 * per)
    assert small.chunk == 3
    small.close()
    ref = _run(wl, obj, I, dev)
    rc = _check(wl, obj, I, dev, ckpt_every=L, workspace_bytes=3 * per)
    assert abs(rc[0] - ref[0]) <= 1e-6 * abs(ref[0])
    assert rel_l2(rc[1], ref[1]) <= 2e-6 and rel_l2(rc[2], ref[2]) <= 2e-6


@pytest.mark.parametrize("M,S,L", [(96, 7, 3), (48, 5, 2), (192, 4, 1)])
def test_recompute_mode_generic_windows(dev, M, S, L):
    """The generic-window path in recompute mode: the same forward and adjoint
    operations in the same order as when every wave is kept, so the loss and
    both gradients are bit-identical; the workspace holds K - 2 checkpoints,
    one segment's waves and exit-wave gradients, the parked state, the wave
    buffer and the probe gradient."""
    wl = synth.workload_random(M, S, 2, 3, 9, seed=60 + M + S, amp_jitter=0.1)
    I = (measurements(wl) * 1.3).astype(np.float32)
    obj = start_object(wl, "perturbed", 8)
    ref = _run(wl, obj, I, dev)
    rc = _check(wl, obj, I, dev, ckpt_every=L)
    assert rc[0] == ref[0] and np.array_equal(rc[1], ref[1]) and np.array_equal(rc[2], ref[2])
    p_rc = _plan(wl, dev, ckpt_every=L)
    K = -(-S // L)
    per = M * M * 8
    assert p_rc.workspace_bytes // wl.N == (K + 2 * L + 1) * per + 8
    p_rc.close()


def test_recompute_interval_auto(dev):
    """ckpt_every = 'auto' keeps K = ceil(sqrt(S)) checkpoints, interval
    ceil(S / K) (S = 10: K = 4, L = 3): the same plan, and the same bits, as
    that interval given explicitly."""
    wl = synth.workload_random(64, 10, 2, 3, 9, seed=77, amp_jitter=0.1)
    I = (measurements(wl) * 1.3).astype(np.float32)
    obj = start_object(wl, "perturbed", 7)
    auto, expl = _plan(wl, dev, ckpt_every="auto"), _plan(wl, dev, ckpt_every=3)
    assert auto.workspace_bytes == expl.workspace_bytes < _plan(wl, dev).workspace_bytes
    auto.close()
    expl.close()
    a = _run(wl, obj, I, dev, ckpt_every="auto")
    b = _run(wl, obj, I, dev, ckpt_every=3)
    assert a[0] == b[0] and np.array_equal(a[1], b[1]) and np.array_equal(a[2], b[2])


def test_recompute_mode_multislice_subset(dev):
    wl = synth.workload_multislice()
    wl.pos = wl.pos[::9]
    I = measurements(wl, counts_seed=1002)
    obj = start_object(wl, "perturbed", 2)
    ref = _run(wl, obj, I, dev)
    rc = _check(wl, obj, I, dev, fp32_floor=True, ckpt_every=4)
    assert rc[0] == ref[0] and rel_l2(rc[1], ref[1]) <= 2e-6 and rel_l2(rc[2], ref[2]) <= 2e-6


# ------------------------------------------------ BF16 hi/lo split on tcgen05

TOL_BF16X3 = 2e-4  # rel-L2 bound of the BF16-split path against the FP64 oracle


# The BF16 hi + lo split represents each operand to about 2^-17; every
# transform of the chain adds that error, which the amplitude residual then
# amplifies, so the 2e-4 bar holds for one or two slices and the error grows
# roughly 5e-5 per slice beyond (measured: S = 5 -> 2.4e-4 / 3.0e-4, S = 16 ->
# 5.4e-4 / 1.1e-3 on gO / gP).  The FP16 split (22 bits) meets 2e-4 at 16 slices.
BF16X3_DEEP_BAR = {5: 4e-4, 16: 2e-3}


@pytest.mark.parametrize("S,ny,nx,step", [(1, 2, 3, 21), (2, 3, 2, 17), (5, 2, 2, 25)])
def test_bf16x3_random_problems(dev, S, ny, nx, step):
    wl = synth.workload_random(128, S, ny, nx, step, seed=60 + S, amp_jitter=0.15)
    I = (measurements(wl) * 1.2).astype(np.float32)
    _check(wl, start_object(wl, "perturbed", 7), I, dev, tol=BF16X3_DEEP_BAR.get(S, TOL_BF16X3),
           precision="bf16x3")


def test_bf16x3_forward(dev):
    wl = synth.workload_random(128, 4, 2, 2, 17, seed=61, amp_jitter=0.1)
    Psi = orc.forward(c64(wl.probe), c64(wl.obj), wl.pos, propagator(wl))
    plan = _plan(wl, dev, precision="bf16x3")
    psi, inten = plan.forward(to_dev(wl.pos, torch.int32, dev), to_dev(wl.probe, torch.complex64, dev),
                              to_dev(wl.obj, torch.complex64, dev), want_psi=True, want_intensity=True)
    torch.cuda.synchronize()
    e = rel_l2(psi.cpu().numpy(), Psi)
    print(f"bf16x3 forward rel-L2 {e:.2e}")
    assert e <= TOL_BF16X3
    plan.status()


def test_bf16x3_multislice_workload(dev):
    """The 16-slice workload (every 4th position) at a perturbed start."""
    wl = synth.workload_multislice()
    wl.pos = wl.pos[::4]
    I = measurements(wl, counts_seed=1002)
    _check(wl, start_object(wl, "perturbed", 2), I, dev, tol=BF16X3_DEEP_BAR[16], precision="bf16x3")


def test_bf16x3_rejects_other_windows(dev):
    from paper_2205_06327_gb300 import api
    from paper_2205_06327_gb300._lib import PTYCHO_ERR_UNSUPPORTED, PtychoError
    with pytest.raises(PtychoError) as e:
        api.Plan(api.Geometry(64, 2, 200, 200, 4), dev, precision="bf16x3")
    assert e.value.code == PTYCHO_ERR_UNSUPPORTED


TOL_FP16X3 = 2e-4


def test_split_product_wait_timeout_is_reported(dev):
    """The split-product kernel's bounded wait on the tensor core: with
    PTYCHO_FLAG_SELFTEST_TIMEOUT it issues no MMAs and waits anyway, so the
    wait expires (about 1 s), the block releases tensor memory and returns,
    and the plan's status reports PTYCHO_ERR_TIMEOUT.  The context stays
    usable: a normal evaluation afterwards matches the oracle."""
    import ctypes as C

    from paper_2205_06327_gb300 import _lib
    wl = synth.workload_random(128, 2, 1, 1, 9, seed=61)
    I = (measurements(wl) * 1.1).astype(np.float32)
    lib = _lib.load()
    p = _lib.PtychoParams(M=wl.M, S=wl.S, H=wl.H, W=wl.W, N=wl.N, lambda_A=wl.lambda_A, dz_A=wl.dz_A,
                          pixel_A=wl.pixel_A, precision=_lib.PTYCHO_FP16X3,
                          flags=_lib.PTYCHO_FLAG_ASYNC_CHECK | _lib.PTYCHO_FLAG_SELFTEST_TIMEOUT)
    h = C.c_void_p()
    assert lib.ptycho_plan_create(C.byref(h), C.byref(p)) == _lib.PTYCHO_OK
    pos, probe = to_dev(wl.pos, torch.int32, dev), to_dev(wl.probe, torch.complex64, dev)
    obj, meas = to_dev(wl.obj, torch.complex64, dev), to_dev(I, torch.float32, dev)
    loss = torch.zeros((), dtype=torch.float64, device=dev)
    rc = lib.ptycho_loss_grad(h, pos.data_ptr(), probe.data_ptr(), obj.data_ptr(), meas.data_ptr(),
                              loss.data_ptr(), None, None, torch.cuda.current_stream(dev).cuda_stream)
    assert rc == _lib.PTYCHO_OK
    torch.cuda.synchronize()
    assert lib.ptycho_plan_status(h) == _lib.PTYCHO_ERR_TIMEOUT
    assert lib.ptycho_plan_destroy(h) == _lib.PTYCHO_OK
    _check(wl, wl.obj, I, dev, tol=2e-4, precision="fp16x3")


@pytest.mark.parametrize("S", [1, 5])
def test_fp16x3_random_problems(dev, S):
    wl = synth.workload_random(128, S, 2, 3, 19, seed=70 + S, amp_jitter=0.15)
    I = (measurements(wl) * 1.2).astype(np.float32)
    _check(wl, start_object(wl, "perturbed", 7), I, dev, tol=TOL_FP16X3, precision="fp16x3")


def test_split_precision_memory_bounded_by_the_workspace_cap(dev):
    """The split precisions keep every wave (no recompute mode), so their
    memory is bounded by the workspace cap through chunking: with room for
    three positions, 12 positions run in chunks of 3 and give the unchunked
    results to reassociation of the chunk sums, within the split bar."""
    wl = synth.workload_random(128, 3, 3, 4, 13, seed=71, amp_jitter=0.1)
    I = (measurements(wl) * 1.2).astype(np.float32)
    obj = start_object(wl, "perturbed", 8)
    per = (2 * wl.S) * 128 * 128 * 8 + 8
    small = _plan(wl, dev, precision="fp16x3", workspace_bytes=3 * per)
    assert small.chunk == 3 and small.workspace_bytes <= 3 * per
    small.close()
    ref = _run(wl, obj, I, dev, precision="fp16x3")
    chunked = _check(wl, obj, I, dev, tol=TOL_FP16X3, precision="fp16x3", workspace_bytes=3 * per)
    assert abs(chunked[0] - ref[0]) <= 1e-6 * abs(ref[0])
    assert rel_l2(chunked[1], ref[1]) <= 1e-6 and rel_l2(chunked[2], ref[2]) <= 1e-6


def test_fp16x3_multislice_workload(dev):
    """The split-precision workload at full size: all 576 positions, 16 slices."""
    wl = synth.workload_multislice()
    I = measurements(wl, counts_seed=1002)
    _check(wl, start_object(wl, "perturbed", 2), I, dev, tol=TOL_FP16X3, precision="fp16x3")


# ------------------------------------------- generic windows (batched FFT path)

@pytest.mark.parametrize("M,S,ny,nx,step", [(96, 1, 2, 3, 13), (96, 3, 2, 2, 17), (192, 2, 2, 2, 31),
                                             (256, 3, 2, 2, 37), (48, 4, 3, 3, 7)])
def test_generic_windows(dev, M, S, ny, nx, step):
    wl = synth.workload_random(M, S, ny, nx, step, seed=90 + M + S, amp_jitter=0.15)
    I = (measurements(wl) * 1.2).astype(np.float32)
    _check(wl, start_object(wl, "perturbed", 4), I, dev)


@pytest.mark.parametrize("seed", range(6))
def test_generic_windows_random_shapes(dev, seed):
    """Seeded random windows 2^a 3^b in [12, 324] on the runtime radix
    schedule and the compiled instances (radix mixes of 8, 4, 2, 3), random
    slice counts, rasters and step sizes, every wave kept or recomputed."""
    g = synth.rng(7000 + seed)
    M = int(g.choice([M for M in range(12, 325) if M not in (64, 128) and _smooth(M)]))
    S = int(g.integers(1, 5))
    ny, nx = int(g.integers(1, 4)), int(g.integers(1, 4))
    step = int(g.integers(1, max(2, M // 3)))
    L = int(g.integers(0, S)) if S > 1 else 0
    wl = synth.workload_random(M, S, ny, nx, step, seed=7100 + seed, amp_jitter=0.1)
    I = (measurements(wl) * 1.15).astype(np.float32)
    _check(wl, start_object(wl, "perturbed", seed), I, dev, ckpt_every=L)


def _smooth(M):
    for p in (2, 3):
        while M % p == 0:
            M //= p
    return M == 1


@pytest.mark.parametrize("M,S,ny,nx,step", [(8, 2, 2, 2, 3), (81, 2, 2, 2, 9)])
def test_generic_window_extremes(dev, M, S, ny, nx, step):
    """The smallest window (one radix-8 stage: the first stage reads and the last
    writes the wave) and a pure radix-3 window."""
    wl = synth.workload_random(M, S, ny, nx, step, seed=120 + M, amp_jitter=0.1)
    I = (measurements(wl) * 1.1).astype(np.float32)
    _check(wl, start_object(wl, "perturbed", 6), I, dev)


def test_generic_window_maximum_size(dev):
    """The largest window the path takes, M = 4096 (one line per block, the
    runtime radix schedule 8 8 8 8, the largest shared-memory request)."""
    wl = synth.workload_random(4096, 1, 1, 1, 8, seed=120 + 4096, amp_jitter=0.1)
    I = (measurements(wl) * 1.1).astype(np.float32)
    _check(wl, start_object(wl, "perturbed", 6), I, dev)


def test_generic_window_forward_and_chunks(dev):
    """Forward far field, and a workspace cap that splits the positions into chunks."""
    wl = synth.workload_random(96, 2, 3, 4, 11, seed=97, amp_jitter=0.1)
    Psi = orc.forward(c64(wl.probe), c64(wl.obj), wl.pos, propagator(wl))
    plan = _plan(wl, dev)
    psi, _ = plan.forward(to_dev(wl.pos, torch.int32, dev), to_dev(wl.probe, torch.complex64, dev),
                          to_dev(wl.obj, torch.complex64, dev))
    torch.cuda.synchronize()
    assert rel_l2(psi.cpu().numpy(), Psi) <= TOL_FP32
    I = (np.abs(Psi) ** 2 * 0.9).astype(np.float32)
    per = (2 * wl.S - 1 + 1) * 96 * 96 * 8 + 96 * 96 * 8 + 8
    ref = _run(wl, start_object(wl, "perturbed", 1), I, dev)
    chunked = _run(wl, start_object(wl, "perturbed", 1), I, dev, workspace_bytes=5 * per)
    assert abs(chunked[0] - ref[0]) <= 1e-12 * abs(ref[0])
    assert rel_l2(chunked[1], ref[1]) <= 1e-6 and rel_l2(chunked[2], ref[2]) <= 1e-6


def test_paper_scale_window_1024(dev):
    """The paper's detector size (Table I: 1024^2 per position), two slices, two positions."""
    wl = synth.workload_random(1024, 2, 1, 2, 200, seed=98, amp_jitter=0.1)
    I = (measurements(wl) * 1.1).astype(np.float32)
    _check(wl, start_object(wl, "perturbed", 2), I, dev)


@pytest.mark.slow
def test_paper_scale_window_1024_100_slices_recompute(dev):
    """Table I's shape per position: 1024^2 windows through 100 slices, in
    recompute mode (auto: 10 checkpoints, segments of 10), two positions,
    against the FP64 oracle.  The 100-slice chain of 1024^2 transforms sits at
    the FP32 rounding floor (the far field carries about 1e-5 of rounding,
    which the amplitude residual amplifies in the loss and the gradients), so
    the bars are the plain-FP32 model's errors on the same inputs."""
    wl = synth.workload_paper_scale(100, 2)
    h = propagator(wl)
    obj = c64(wl.obj)
    I = (orc.intensities(c64(wl.probe), obj, wl.pos, h) * 1.1).astype(np.float32)
    plan = _plan(wl, dev, ckpt_every="auto")
    per = 1024 * 1024 * 8
    assert plan.workspace_bytes // wl.N == (10 + 2 * 10 + 1) * per + 8
    plan.close()
    _check(wl, obj, I, dev, fp32_floor=True, ckpt_every="auto")


def test_generic_window_more_positions_than_a_chunk(dev):
    """M = 256 keeps at most 128 waves per chunk (L2-sized): 130 positions take two
    chunks in both the forward model and the gradient."""
    wl = synth.workload_random(256, 1, 10, 13, 2, seed=99, amp_jitter=0.1)
    assert wl.N == 130
    Psi = orc.forward(c64(wl.probe), c64(wl.obj), wl.pos, propagator(wl))
    plan = _plan(wl, dev)
    assert plan.chunk < wl.N
    _, inten = plan.forward(to_dev(wl.pos, torch.int32, dev), to_dev(wl.probe, torch.complex64, dev),
                            to_dev(wl.obj, torch.complex64, dev), want_psi=False, want_intensity=True)
    torch.cuda.synchronize()
    assert rel_l2(inten.cpu().numpy(), np.abs(Psi) ** 2) <= TOL_FP32
    I = (np.abs(Psi) ** 2 * 1.1).astype(np.float32)
    _check(wl, start_object(wl, "perturbed", 3), I, dev)


def test_generic_windows_plans_coexist(dev):
    """Plans for different generic windows created first, used afterwards (the
    FFT kernels' shared-memory limit is shared by all plans)."""
    wls = [synth.workload_random(M, 1, 2, 2, 9, seed=100 + M) for M in (256, 96)]
    plans = [_plan(wl, dev) for wl in wls]
    for wl, plan in zip(wls, plans):
        I = (measurements(wl) * 1.2).astype(np.float32)
        loss, _, _ = plan.loss_grad(to_dev(wl.pos, torch.int32, dev), to_dev(wl.probe, torch.complex64, dev),
                                    to_dev(wl.obj, torch.complex64, dev), to_dev(I, torch.float32, dev))
        L = orc.loss(c64(wl.probe), c64(wl.obj), wl.pos, I.astype(np.float64), propagator(wl))
        assert abs(loss.item() - L) <= TOL_FP32 * L
