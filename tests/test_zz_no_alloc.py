"""ptycho_loss_grad_noalloc through the C-ABI.

The allocation-free entry point serves callers that cannot call cudaMalloc:
code inside a custom device allocator or memory-pool callback (a cudaMalloc
there would re-enter the allocator), or a process whose device memory is
fixed after start-up.  It runs the same kernels out of one static 64 MiB
device array, in smaller chunks, so its results must match the plan-based
entry point to within reassociation of the chunked sums, and the FP64 oracle
within the FP32 path's tolerance.  Two calls in a row on different inputs
check that nothing stale from the previous call leaks into the next (the
array keeps its contents between calls), and the device's free memory must
not change across those calls.

Collected last on purpose (file name), so a run that stops at the first
failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

from oracle import ptycho_oracle as orc
from paper_2205_06327_gb300 import synth
from tests.helpers import TOL_FP32, c64, measurements, propagator, rel_l2, start_object, to_dev

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5  # the parity tolerance of the FP32 path; here both sides are the same kernels


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda", 0)


def _lib():
    from paper_2205_06327_gb300 import _lib
    return _lib, _lib.load()


def _inputs(wl, obj, I, dev):
    return (to_dev(wl.pos, torch.int32, dev), to_dev(wl.probe, torch.complex64, dev),
            to_dev(obj, torch.complex64, dev), to_dev(I, torch.float32, dev))


def _params(wl, N=None):
    L, _ = _lib()
    return L.PtychoParams(M=wl.M, S=wl.S, H=wl.H, W=wl.W, N=wl.N if N is None else N, lambda_A=wl.lambda_A,
                          dz_A=wl.dz_A, pixel_A=wl.pixel_A)


def _outputs(wl, dev):
    gO = torch.full((wl.S, wl.H, wl.W), 7.0, dtype=torch.complex64, device=dev)  # stale values
    gP = torch.full((wl.M, wl.M), 7.0, dtype=torch.complex64, device=dev)
    loss = torch.full((), -1.0, dtype=torch.float64, device=dev)
    return loss, gO, gP


def _call(p, pos, probe, obj, I, loss_ptr, gO, gP, dev):
    _, lib = _lib()
    stream = torch.cuda.current_stream(dev).cuda_stream
    return lib.ptycho_loss_grad_noalloc(C.byref(p), pos.data_ptr(), probe.data_ptr(), obj.data_ptr(),
                                        I.data_ptr(), loss_ptr, gO.data_ptr() if gO is not None else None,
                                        gP.data_ptr() if gP is not None else None, stream)


def _with_plan(wl, pos, probe, obj, I, dev):
    from paper_2205_06327_gb300 import api
    plan = api.Plan(api.Geometry(wl.M, wl.S, wl.H, wl.W, wl.N, wl.lambda_A, wl.dz_A, wl.pixel_A), dev)
    loss, gO, gP = plan.loss_grad(pos, probe, obj, I)
    torch.cuda.synchronize()
    out = loss.item(), gO.cpu().numpy(), gP.cpu().numpy()
    plan.close()
    return out


def test_noalloc_matches_plan_entry_point_two_calls_without_allocating(dev):
    # 16 slices of 128^2: 4 MiB of scratch per position, so the static array
    # runs the 48 positions in several chunks
    L, _ = _lib()
    wl = synth.workload_multislice()
    wl.pos = wl.pos.reshape(24, 24, 2)[6:12, 4:12].reshape(-1, 2).copy()
    I = measurements(wl, counts_seed=1002)
    calls = []
    for call, kind in enumerate(["perturbed", "truth"]):
        obj = start_object(wl, kind, 3 + call)
        calls.append((_inputs(wl, obj, I, dev), _outputs(wl, dev)))
    p = _params(wl)
    # device set-up, and the first use of every kernel (lazy module loading)
    assert _call(p, *calls[0][0], calls[0][1][0].data_ptr(), calls[0][1][1], calls[0][1][2], dev) == L.PTYCHO_OK
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    for args, (loss, gO, gP) in calls:
        assert _call(p, *args, loss.data_ptr(), gO, gP, dev) == L.PTYCHO_OK
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0, "the allocation-free call changed free device memory"
    for args, (loss, gO, gP) in calls:
        l0, o0, p0 = _with_plan(wl, *args, dev)
        assert abs(loss.item() - l0) <= TOL * abs(l0)
        assert rel_l2(gO.cpu().numpy(), o0) <= TOL and rel_l2(gP.cpu().numpy(), p0) <= TOL


def test_noalloc_single_slice_against_oracle_host_loss_and_null_gradients(dev):
    """M = 64, one slice, against the FP64 oracle directly; the loss written to
    a host double; then a loss-only call with both gradient pointers NULL."""
    L, _ = _lib()
    wl = synth.workload_single_slice()
    I = measurements(wl)
    obj = start_object(wl, "perturbed", 5)
    args = _inputs(wl, obj, I, dev)
    host_loss = C.c_double(-1.0)
    _, gO, gP = _outputs(wl, dev)
    assert _call(_params(wl), *args, C.addressof(host_loss), gO, gP, dev) == L.PTYCHO_OK
    Lr, gOr, gPr = orc.loss_grad(c64(wl.probe), c64(obj), wl.pos, I.astype(np.float64), propagator(wl))
    assert abs(host_loss.value - Lr) <= TOL_FP32 * abs(Lr)
    assert rel_l2(gO.cpu().numpy(), gOr) <= TOL_FP32 and rel_l2(gP.cpu().numpy(), gPr) <= TOL_FP32
    only = C.c_double(-1.0)
    assert _call(_params(wl), *args, C.addressof(only), None, None, dev) == L.PTYCHO_OK
    assert only.value == host_loss.value


def test_noalloc_zero_positions_and_window_outside(dev):
    L, _ = _lib()
    wl = synth.workload_random(64, 2, 2, 2, 9, seed=8)
    I = measurements(wl)
    args = _inputs(wl, wl.obj, I, dev)
    loss, gO, gP = _outputs(wl, dev)
    assert _call(_params(wl, N=0), *args, loss.data_ptr(), gO, gP, dev) == L.PTYCHO_OK
    torch.cuda.synchronize()
    assert loss.item() == 0.0
    assert not gO.abs().any().item() and not gP.abs().any().item()
    bad = args[0].clone()
    bad[1, 1] = wl.W - wl.M + 1  # one window one pixel past the right edge
    loss, gO, gP = _outputs(wl, dev)
    rc = _call(_params(wl), bad, *args[1:], loss.data_ptr(), gO, gP, dev)
    assert rc == L.PTYCHO_ERR_POSITION
    assert np.isfinite(loss.item()) and loss.item() >= 0.0


def test_noalloc_rejects_misaligned_arrays_and_problems_beyond_the_scratch(dev):
    L, lib = _lib()
    wl = synth.workload_random(128, 2, 1, 1, 1, seed=5)
    pos, probe, obj, I = _inputs(wl, wl.obj, measurements(wl), dev)
    loss = torch.zeros(2, dtype=torch.float64, device=dev)
    p = _params(wl)
    # a float pointer 4 bytes into the probe: rejected before any launch
    rc = lib.ptycho_loss_grad_noalloc(C.byref(p), pos.data_ptr(), probe.data_ptr() + 4, obj.data_ptr(),
                                      I.data_ptr(), loss.data_ptr(), None, None, None)
    assert rc == L.PTYCHO_ERR_ARG
    rc = lib.ptycho_loss_grad_noalloc(C.byref(p), pos.data_ptr(), probe.data_ptr(), obj.data_ptr(),
                                      I.data_ptr(), loss.data_ptr() + 4, None, None, None)
    assert rc == L.PTYCHO_ERR_ARG
    big = L.PtychoParams(M=128, S=400, H=wl.H, W=wl.W, N=1, lambda_A=0.0251, dz_A=2.0, pixel_A=0.1)
    rc = lib.ptycho_loss_grad_noalloc(C.byref(big), pos.data_ptr(), probe.data_ptr(), obj.data_ptr(),
                                      I.data_ptr(), loss.data_ptr(), None, None, None)
    assert rc == L.PTYCHO_ERR_UNSUPPORTED
