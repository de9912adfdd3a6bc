"""Several problems advanced together under one captured CUDA graph per
iteration, and the measured accumulation-tile choice."""
import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from paper_2205_06327_gb300 import synth
from tests.helpers import c64, measurements, propagator, rel_l2, start_object, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda", 0)


def _problems(dev, specs):
    from paper_2205_06327_gb300 import api
    from paper_2205_06327_gb300.multi import Problem
    out, host = [], []
    for k, (M, S, ny, nx, step) in enumerate(specs):
        wl = synth.workload_random(M, S, ny, nx, step, seed=500 + k, amp_jitter=0.1)
        I = (measurements(wl) * 1.1).astype(np.float32)
        obj = start_object(wl, "perturbed", k)
        g = api.Geometry(wl.M, wl.S, wl.H, wl.W, wl.N, wl.lambda_A, wl.dz_A, wl.pixel_A)
        out.append(Problem(g, to_dev(wl.pos, torch.int32, dev), to_dev(wl.probe, torch.complex64, dev),
                           to_dev(obj, torch.complex64, dev), to_dev(I, torch.float32, dev)))
        host.append((wl, obj, I))
    return out, host


SPECS = [(64, 2, 3, 3, 9), (128, 3, 2, 2, 21), (64, 1, 4, 2, 11), (128, 1, 2, 3, 19)]


def test_graph_replay_matches_eager_and_oracle(dev):
    from paper_2205_06327_gb300.multi import MultiProblem
    a_o, a_p = 2e-3, 1e-5
    probs, host = _problems(dev, SPECS)
    eager, _ = _problems(dev, SPECS)
    mp = MultiProblem(probs, dev)
    me = MultiProblem(eager, dev)
    mp.capture(a_o, a_p, warmup=1)   # warm-up = iteration 1, the capture itself runs nothing
    me.step_all(a_o, a_p)
    mp.run(2)                        # iterations 2 and 3
    me.step_all(a_o, a_p)
    me.step_all(a_o, a_p)
    torch.cuda.synchronize()
    mp.check_status()
    for p, q in zip(probs, eager):   # graph replay == eager, bit for bit
        assert torch.equal(p.obj, q.obj) and torch.equal(p.probe, q.probe)
    assert torch.equal(mp.loss, me.loss)
    for p, (wl, obj, I) in zip(probs, host):  # three FP64 oracle steps
        P, O = c64(wl.probe), c64(obj)
        h = propagator(wl)
        for _ in range(3):
            P, O, _, _ = orc.step(P, O, wl.pos, I.astype(np.float64), h, a_o, a_p)
        assert rel_l2(p.obj.cpu().numpy(), O) <= 1e-6 and rel_l2(p.probe.cpu().numpy(), P) <= 1e-6
    mp.close()
    me.close()


# Every window class of the batched workload (64, 96, 128, 192, 256), slices
# up to 24, and a workspace small enough that the generic-window problems run
# their positions in several chunks.
EVERY_WINDOW = [(64, 24, 2, 2, 9), (96, 5, 2, 3, 9), (128, 16, 2, 2, 21), (192, 3, 2, 2, 13),
                (256, 6, 2, 3, 11), (64, 1, 3, 3, 9), (128, 2, 2, 2, 19)]


def test_graph_replay_every_window_class_against_oracle(dev):
    """Seven problems covering every window class under captured CUDA graphs.
    (1) One captured multi-problem loss-and-gradient call, replayed: every
    problem's loss and gradients against the FP64 oracle, element by element,
    at 1e-5 (for 16 slices and more, the FP32 rounding floor measured by the
    single-precision model).  (2) Three gradient-descent iterations, the first
    eager and two replayed from one captured graph: the iterates equal three
    eager iterations bit for bit and three FP64 oracle steps to 1e-6."""
    from paper_2205_06327_gb300 import _lib
    from paper_2205_06327_gb300.api import _stream_handle
    from paper_2205_06327_gb300.multi import MultiProblem
    from tests.helpers import fp32_chain_loss_grad
    probs, host = _problems(dev, EVERY_WINDOW)
    eager, _ = _problems(dev, EVERY_WINDOW)
    ws = len(probs) * (14 << 20)
    mp, me = MultiProblem(probs, dev, workspace_bytes=ws), MultiProblem(eager, dev, workspace_bytes=ws)
    assert any(pl.chunk < p.geom.N for pl, p in zip(mp.plans, probs) if p.geom.M in (96, 192, 256))

    # (1) gradients from a replayed graph
    grads = [(torch.empty_like(p.obj), torch.empty_like(p.probe)) for p in probs]
    arr = mp._entries(grads)
    lib = mp.plans[0].lib
    call = lambda: _lib.check(lib.ptycho_multi_loss_grad(arr, len(probs), _stream_handle(dev)))
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(side):
        call()  # warm-up: every workspace allocated before capture
    torch.cuda.current_stream(dev).wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, capture_error_mode="relaxed"):
        call()
    for go, gp in grads:
        go.zero_()
        gp.zero_()
    mp.loss.zero_()
    graph.replay()
    torch.cuda.synchronize()
    mp.check_status()
    for k, ((go, gp), (wl, obj, I)) in enumerate(zip(grads, host)):
        P, O, h = c64(wl.probe), c64(obj), propagator(wl)
        L, gO, gP = orc.loss_grad(P, O, wl.pos, I.astype(np.float64), h)
        bar_l = bar_o = bar_p = 1e-5
        if wl.S >= 16:
            lf, fo, fp = fp32_chain_loss_grad(wl.probe, obj, wl.pos, I, h)
            bar_l, bar_o, bar_p = (max(bar_l, 1.5 * abs(lf - L) / L), max(bar_o, 1.5 * rel_l2(fo, gO)),
                                   max(bar_p, 1.5 * rel_l2(fp, gP)))
        el = abs(mp.loss[k].item() - L) / L
        eo, ep = rel_l2(go.cpu().numpy(), gO), rel_l2(gp.cpu().numpy(), gP)
        print(f"M={wl.M} S={wl.S} N={wl.N}: loss {el:.2e} gO {eo:.2e} (bar {bar_o:.1e}) gP {ep:.2e} "
              f"(bar {bar_p:.1e})")
        assert el <= bar_l and eo <= bar_o and ep <= bar_p
    del graph

    # (2) iterates from a replayed step graph
    a_o, a_p = 2e-3, 1e-5
    mp.capture(a_o, a_p, warmup=1)
    mp.run(2)
    for _ in range(3):
        me.step_all(a_o, a_p)
    torch.cuda.synchronize()
    mp.check_status()
    for p, q, (wl, obj, I) in zip(probs, eager, host):
        assert torch.equal(p.obj, q.obj) and torch.equal(p.probe, q.probe)
        P, O, h = c64(wl.probe), c64(obj), propagator(wl)
        for _ in range(3):
            P, O, _, _ = orc.step(P, O, wl.pos, I.astype(np.float64), h, a_o, a_p)
        assert rel_l2(p.obj.cpu().numpy(), O) <= 1e-6 and rel_l2(p.probe.cpu().numpy(), P) <= 1e-6
    mp.close()
    me.close()


def test_multi_loss_grad_matches_single_calls(dev):
    """One multi-problem call (a generic window among the problems) gives the
    single-problem results bit for bit."""
    from paper_2205_06327_gb300.multi import MultiProblem
    specs = SPECS + [(96, 2, 2, 2, 13)]
    probs, _ = _problems(dev, specs)
    mp = MultiProblem(probs, dev)
    loss, grads = mp.loss_grad_all()
    torch.cuda.synchronize()
    mp.check_status()
    for i, (p, plan) in enumerate(zip(probs, mp.plans)):
        l1, go, gp = plan.loss_grad(p.pos, p.probe, p.obj, p.meas)
        torch.cuda.synchronize()
        assert l1.item() == loss[i].item()
        assert torch.equal(go, grads[i][0]) and torch.equal(gp, grads[i][1])
    mp.close()


def test_multi_call_many_problems_several_chunks_matches_single_calls(dev):
    """Eighteen register-resident problems (more than one multi-problem chain
    launch takes) whose positions run in several chunks: the multi-problem
    call launches each round's chains of all problems together and must still
    give every problem's single-call results bit for bit."""
    from paper_2205_06327_gb300.multi import MultiProblem
    specs = [(64 if k % 2 else 128, 1 + k % 3, 2, 2 + k % 3, 9 + k) for k in range(18)]
    probs, _ = _problems(dev, specs)
    # about three positions per chunk for the deepest 128-window problems
    mp = MultiProblem(probs, dev, workspace_bytes=18 * (3 * 6 * 128 * 128 * 8))
    assert max(-(-p.geom.N // pl.chunk) for p, pl in zip(probs, mp.plans)) >= 2
    loss, grads = mp.loss_grad_all()
    torch.cuda.synchronize()
    mp.check_status()
    for i, (p, plan) in enumerate(zip(probs, mp.plans)):
        l1, go, gp = plan.loss_grad(p.pos, p.probe, p.obj, p.meas)
        torch.cuda.synchronize()
        assert l1.item() == loss[i].item()
        assert torch.equal(go, grads[i][0]) and torch.equal(gp, grads[i][1])
    mp.close()


def test_multi_call_argument_errors(dev):
    from paper_2205_06327_gb300 import _lib
    from paper_2205_06327_gb300.multi import MultiProblem
    probs, _ = _problems(dev, SPECS[:2])
    mp = MultiProblem(probs, dev)
    lib = mp.plans[0].lib
    arr = mp._entries()
    arr[1].plan = arr[0].plan  # two entries sharing a plan
    assert lib.ptycho_multi_step(arr, 2, 1e-3, 0.0, None) == _lib.PTYCHO_ERR_ARG
    assert b"share a plan" in lib.ptycho_last_error()
    arr = mp._entries()
    host_loss = (_lib.C.c_double * 1)()
    arr[1].loss_out = _lib.C.addressof(host_loss)  # host pointer: the call never synchronises
    assert lib.ptycho_multi_loss_grad(arr, 2, None) == _lib.PTYCHO_ERR_ARG
    assert b"problem 1" in lib.ptycho_last_error()
    assert lib.ptycho_multi_step(arr, -1, 1e-3, 0.0, None) == _lib.PTYCHO_ERR_ARG
    mp.close()


def test_unsupported_window_is_refused(dev):
    from paper_2205_06327_gb300 import api
    from paper_2205_06327_gb300.multi import MultiProblem, Problem, supported
    assert supported(64) and supported(128) and supported(96) and supported(192) and supported(256)
    assert not supported(100) and supported(128, "bf16x3") and not supported(96, "fp16x3")
    g = api.Geometry(100, 1, 200, 200, 1)
    z = torch.zeros(1, device=dev)
    with pytest.raises(ValueError):
        MultiProblem([Problem(g, z, z, z, z)], dev)


def test_autotuner_picks_and_caches_a_tile(dev, tmp_path, monkeypatch):
    from paper_2205_06327_gb300 import api, autotune
    monkeypatch.setenv("PTYCHO_GB300_CACHE", str(tmp_path))
    wl = synth.workload_random(64, 2, 4, 4, 6, seed=77)
    I = measurements(wl)
    g = api.Geometry(wl.M, wl.S, wl.H, wl.W, wl.N, wl.lambda_A, wl.dz_A, wl.pixel_A)
    args = (to_dev(wl.pos, torch.int32, dev), to_dev(wl.probe, torch.complex64, dev),
            to_dev(wl.obj, torch.complex64, dev), to_dev(I, torch.float32, dev))
    tile = autotune.tune_tile(g, *args, device=dev, candidates=((16, 16), (32, 32)))
    assert tile in ((16, 16), (32, 32))
    assert autotune.tune_tile(g, *args, device=dev, candidates=()) == tile  # from the cache
    assert (tmp_path / "autotune.json").exists()


@pytest.mark.parametrize("batch", [1, 3, 7])
def test_sequential_gd_matches_oracle_steps(dev, batch):
    """Algorithm 1's sequential update (batch = 1) and mini-batches: one epoch of
    updates after every batch, against the same sequence of FP64 oracle steps."""
    from paper_2205_06327_gb300 import api
    from paper_2205_06327_gb300.sgd import SequentialGD
    wl = synth.workload_random(64, 2, 2, 4, 10, seed=88, amp_jitter=0.1)
    I = (measurements(wl) * 1.1).astype(np.float32)
    obj0 = start_object(wl, "perturbed", 3)
    g = api.Geometry(wl.M, wl.S, wl.H, wl.W, wl.N, wl.lambda_A, wl.dz_A, wl.pixel_A)
    a_o, a_p = 5e-3, 2e-5
    sgd = SequentialGD(g, batch, dev)
    P = to_dev(wl.probe, torch.complex64, dev)
    O = to_dev(obj0, torch.complex64, dev)
    losses = sgd.epoch(to_dev(wl.pos, torch.int32, dev), P, O, to_dev(I, torch.float32, dev), a_o, a_p)
    torch.cuda.synchronize()
    Pr, Or = c64(wl.probe), c64(obj0)
    h = propagator(wl)
    ref_losses = []
    for i0 in range(0, wl.N, batch):
        sl = slice(i0, min(wl.N, i0 + batch))
        Pr, Or, F0, _ = orc.step(Pr, Or, wl.pos[sl], I[sl].astype(np.float64), h, a_o, a_p)
        ref_losses.append(F0)
    assert np.allclose(losses.cpu().numpy(), ref_losses, rtol=1e-5)
    assert rel_l2(O.cpu().numpy(), Or) <= 1e-6 and rel_l2(P.cpu().numpy(), Pr) <= 1e-6
    sgd.close()


def test_sequential_gd_convergence_by_batch(dev):
    """Loss against epochs for Algorithm 1's per-position updates, mini-batches and
    the full batch at the same step size (the paper's question of how often to
    update, Sec. VI-F, Fig. 9): every schedule lowers the cost every epoch, and at this
    small step the schedules agree to first order (within 1 %)."""
    from paper_2205_06327_gb300 import api
    from paper_2205_06327_gb300.sgd import SequentialGD
    wl = synth.workload_random(64, 3, 4, 4, 10, seed=89, amp_jitter=0.1)
    I = (measurements(wl) * 1.05).astype(np.float32)
    obj0 = start_object(wl, "perturbed", 4)
    g = api.Geometry(wl.M, wl.S, wl.H, wl.W, wl.N, wl.lambda_A, wl.dz_A, wl.pixel_A)
    a_o, a_p = 1e-2, 0.0
    pos, meas = to_dev(wl.pos, torch.int32, dev), to_dev(I, torch.float32, dev)
    full = api.Plan(g, dev)
    curves = {}
    for batch in (1, 4, wl.N):
        sgd = SequentialGD(g, batch, dev)
        P, O = to_dev(wl.probe, torch.complex64, dev), to_dev(obj0, torch.complex64, dev)
        F = [full.loss_grad(pos, P, O, meas, want_obj=False, want_probe=False)[0].item()]
        for _ in range(4):
            sgd.epoch(pos, P, O, meas, a_o, a_p)
            F.append(full.loss_grad(pos, P, O, meas, want_obj=False, want_probe=False)[0].item())
        curves[batch] = F
        sgd.close()
    full.close()
    for batch, F in curves.items():
        print(f"batch {batch:3d}: F per epoch " + " ".join(f"{f:.4e}" for f in F))
        assert all(b < a for a, b in zip(F, F[1:]))
        assert np.allclose(F, curves[wl.N], rtol=1e-2)


# ------------------------------------- Algorithm 1's delayed accumulation (period T)

@pytest.mark.parametrize("T", [1, 3, 5])
def test_delayed_accumulation_matches_oracle_sequence(dev, T):
    """Per-location updates with the accumulated-gradient buffer: after every
    T-th location the buffer is applied as a second update and cleared, and it
    carries over into the next epoch.  Two epochs of 7 locations (so the flushes
    fall at different places in each epoch) against the same sequence of FP64
    oracle gradients."""
    from paper_2205_06327_gb300 import api
    from paper_2205_06327_gb300.sgd import SequentialGD
    wl = synth.workload_random(64, 2, 1, 7, 8, seed=91, amp_jitter=0.1)
    I = (measurements(wl) * 1.1).astype(np.float32)
    obj0 = start_object(wl, "perturbed", 5)
    g = api.Geometry(wl.M, wl.S, wl.H, wl.W, wl.N, wl.lambda_A, wl.dz_A, wl.pixel_A)
    a_o, a_p = 4e-3, 1e-5
    sgd = SequentialGD(g, 1, dev, period=T)
    P = to_dev(wl.probe, torch.complex64, dev)
    O = to_dev(obj0, torch.complex64, dev)
    pos, meas = to_dev(wl.pos, torch.int32, dev), to_dev(I, torch.float32, dev)
    losses = [sgd.epoch(pos, P, O, meas, a_o, a_p).cpu().numpy() for _ in range(2)]
    torch.cuda.synchronize()
    Pr, Or = c64(wl.probe), c64(obj0)
    acc = np.zeros_like(Or)
    h = propagator(wl)
    ref, i = [], 0
    for _ in range(2):
        for k in range(wl.N):
            F0, gO, gP = orc.loss_grad(Pr, Or, wl.pos[k:k + 1], I[k:k + 1].astype(np.float64), h)
            ref.append(F0)
            Or = Or - a_o * gO
            Pr = Pr - a_p * gP
            acc += gO
            i += 1
            if i % T == 0:
                Or = Or - a_o * acc
                acc[:] = 0
    assert np.allclose(np.concatenate(losses), ref, rtol=1e-5)
    assert rel_l2(O.cpu().numpy(), Or) <= 1e-6 and rel_l2(P.cpu().numpy(), Pr) <= 1e-6
    assert rel_l2(sgd.acc.cpu().numpy(), acc) <= 1e-5 if np.any(acc) else not sgd.acc.abs().any().item()
    sgd.close()


def test_delayed_accumulation_period_one_is_a_double_step(dev):
    """With one tile and T = 1 the buffer holds exactly the location's own
    gradient, so each location takes two steps of alpha on the same gradient:
    the same iterates as per-location descent with step 2 alpha."""
    from paper_2205_06327_gb300 import api
    from paper_2205_06327_gb300.sgd import SequentialGD
    wl = synth.workload_random(64, 3, 2, 3, 9, seed=92, amp_jitter=0.1)
    I = (measurements(wl) * 1.1).astype(np.float32)
    obj0 = start_object(wl, "perturbed", 6)
    g = api.Geometry(wl.M, wl.S, wl.H, wl.W, wl.N, wl.lambda_A, wl.dz_A, wl.pixel_A)
    pos, meas = to_dev(wl.pos, torch.int32, dev), to_dev(I, torch.float32, dev)
    out = []
    for period, a in ((1, 3e-3), (0, 6e-3)):
        sgd = SequentialGD(g, 1, dev, period=period)
        P, O = to_dev(wl.probe, torch.complex64, dev), to_dev(obj0, torch.complex64, dev)
        sgd.epoch(pos, P, O, meas, a, 0.0)
        out.append(O.cpu().numpy())
        sgd.close()
    assert rel_l2(out[0], out[1]) <= 1e-6


def test_delayed_accumulation_convergence_by_period(dev):
    """The paper's question of how often to communicate (Sec. VI-F, Fig. 9):
    loss against epochs for T = 1, N/8 and N on a 64-position block of the
    576-position multislice workload (16 slices of 384^2, Poisson data), with
    per-location steps.  Every schedule lowers the cost every epoch."""
    from paper_2205_06327_gb300 import api
    from paper_2205_06327_gb300.sgd import SequentialGD
    wl = synth.workload_multislice()
    wl.pos = wl.pos.reshape(24, 24, 2)[8:16, 8:16].reshape(-1, 2).copy()
    I = measurements(wl, counts_seed=1002)
    obj0 = start_object(wl, "perturbed", 9)
    g = api.Geometry(wl.M, wl.S, wl.H, wl.W, wl.N, wl.lambda_A, wl.dz_A, wl.pixel_A)
    pos, meas = to_dev(wl.pos, torch.int32, dev), to_dev(I, torch.float32, dev)
    full = api.Plan(g, dev)
    _, g0, _ = full.loss_grad(pos, to_dev(wl.probe, torch.complex64, dev), to_dev(obj0, torch.complex64, dev),
                              meas, want_probe=False)
    a = 0.05 / float(g0.abs().max())  # a full-batch step moves O by at most 5 %
    curves = {}
    for T in (1, wl.N // 8, wl.N):
        sgd = SequentialGD(g, 1, dev, period=T)
        P, O = to_dev(wl.probe, torch.complex64, dev), to_dev(obj0, torch.complex64, dev)
        F = [full.loss_grad(pos, P, O, meas, want_obj=False, want_probe=False)[0].item()]
        for _ in range(3):
            sgd.epoch(pos, P, O, meas, a, 0.0)
            F.append(full.loss_grad(pos, P, O, meas, want_obj=False, want_probe=False)[0].item())
        curves[T] = F
        sgd.close()
    full.close()
    for T, F in curves.items():
        print(f"T = {T:3d}: F per epoch " + " ".join(f"{f:.6e}" for f in F))
        assert all(b < a for a, b in zip(F, F[1:])), (T, F)


@pytest.mark.parametrize("T", [1, 3])
def test_delayed_accumulation_matches_the_host_ranks_schedule(dev, T):
    """The GPU's Algorithm 1 (SequentialGD with period T, one tile) against the
    host-rank implementation of the same schedule (halo_passes.appp_epoch on a
    one-tile grid in a one-rank gloo group, with the FP64 oracle's
    per-location gradients): two implementations of the algorithm, one epoch,
    the object's iterates to 1e-6."""
    import os
    import socket

    import torch.distributed as dist

    from paper_2205_06327_gb300 import api
    from paper_2205_06327_gb300 import halo_passes as hp
    from paper_2205_06327_gb300.sgd import SequentialGD
    wl = synth.workload_random(64, 2, 2, 3, 9, seed=93, amp_jitter=0.1)
    I = (measurements(wl) * 1.1).astype(np.float32)
    obj0 = c64(start_object(wl, "perturbed", 7))
    P, h, a = c64(wl.probe), propagator(wl), 3e-3
    g = api.Geometry(wl.M, wl.S, wl.H, wl.W, wl.N, wl.lambda_A, wl.dz_A, wl.pixel_A)
    sgd = SequentialGD(g, 1, dev, period=T)
    O = to_dev(obj0, torch.complex64, dev)
    sgd.epoch(to_dev(wl.pos, torch.int32, dev), to_dev(wl.probe, torch.complex64, dev), O,
              to_dev(I, torch.float32, dev), a, 0.0)
    torch.cuda.synchronize()
    sgd.close()
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        grid = hp.tile_grid(wl.H, wl.W, 1, 1, wl.pos, wl.M)
        me = grid[0][0]
        e = me.ext
        assert (e.y0, e.x0, e.y1, e.x1) == (0, 0, wl.H, wl.W)

        def grad_fn(i, tile):
            _, gOi, _ = orc.position_loss_grad(P, tile.numpy(), wl.pos[i], I[i].astype(np.float64), h)
            gr = torch.zeros_like(tile)
            y, x = int(wl.pos[i][0]), int(wl.pos[i][1])
            gr[:, y:y + wl.M, x:x + wl.M] = torch.from_numpy(gOi)
            return gr

        tile = torch.from_numpy(obj0.copy())
        hp.appp_epoch(tile, torch.zeros_like(tile), grid, me, np.arange(wl.N), grad_fn, a, T)
    finally:
        dist.destroy_process_group()
    assert rel_l2(O.cpu().numpy(), tile.numpy()) <= 1e-6
