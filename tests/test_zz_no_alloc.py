"""ptycho_loss_grad_noalloc through the C-ABI against ptycho_loss_grad.

The allocation-free entry point serves callers that cannot call cudaMalloc
(code inside a custom device allocator or pool callback, or a process whose
device memory is fixed after start-up).  It runs the same kernels out of one
static 64 MiB device array, in smaller chunks, so its results must match the
plan-based entry point to within reassociation of the chunked sums.  Two calls
in a row on different inputs also check that nothing stale from the previous
call leaks into the next (the array keeps its contents between calls).

Collected last on purpose (file name), so a run that stops at the first
failure has already run every other test.
"""
import ctypes as C

import pytest

from paper_2205_06327_gb300 import synth
from tests.helpers import measurements, rel_l2, start_object, to_dev

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


def _inputs(wl, obj, I, dev):
    return (to_dev(wl.pos, torch.int32, dev), to_dev(wl.probe, torch.complex64, dev),
            to_dev(obj, torch.complex64, dev), to_dev(I, torch.float32, dev))


def _noalloc(wl, pos, probe, obj, I, dev):
    from paper_2205_06327_gb300 import _lib
    lib = _lib.load()
    p = _lib.PtychoParams(M=wl.M, S=wl.S, H=wl.H, W=wl.W, N=wl.N, lambda_A=wl.lambda_A, dz_A=wl.dz_A,
                          pixel_A=wl.pixel_A)
    gO = torch.zeros((wl.S, wl.H, wl.W), dtype=torch.complex64, device=dev)
    gP = torch.zeros((wl.M, wl.M), dtype=torch.complex64, device=dev)
    loss = torch.zeros((), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream
    rc = lib.ptycho_loss_grad_noalloc(C.byref(p), pos.data_ptr(), probe.data_ptr(), obj.data_ptr(), I.data_ptr(),
                                      loss.data_ptr(), gO.data_ptr(), gP.data_ptr(), stream)
    assert rc == _lib.PTYCHO_OK, rc
    return loss.item(), gO.cpu().numpy(), gP.cpu().numpy()


def _with_plan(wl, pos, probe, obj, I, dev):
    from paper_2205_06327_gb300 import api
    plan = api.Plan(api.Geometry(wl.M, wl.S, wl.H, wl.W, wl.N, wl.lambda_A, wl.dz_A, wl.pixel_A), dev)
    loss, gO, gP = plan.loss_grad(pos, probe, obj, I)
    torch.cuda.synchronize()
    out = loss.item(), gO.cpu().numpy(), gP.cpu().numpy()
    plan.close()
    return out


def test_noalloc_matches_plan_entry_point_two_calls(dev):
    # 16 slices of 128^2: 4 MiB of scratch per position, so the static array
    # runs the 48 positions in several chunks
    wl = synth.workload_multislice()
    wl.pos = wl.pos.reshape(24, 24, 2)[6:12, 4:12].reshape(-1, 2).copy()
    I = measurements(wl, counts_seed=1002)
    for call, kind in enumerate(["perturbed", "truth"]):
        obj = start_object(wl, kind, 3 + call)
        args = _inputs(wl, obj, I, dev)
        l1, o1, p1 = _noalloc(wl, *args, dev)
        l0, o0, p0 = _with_plan(wl, *args, dev)
        assert abs(l1 - l0) <= TOL * abs(l0)
        assert rel_l2(o1, o0) <= TOL and rel_l2(p1, p0) <= TOL


def test_noalloc_rejects_problems_beyond_the_scratch(dev):
    from paper_2205_06327_gb300 import _lib
    lib = _lib.load()
    wl = synth.workload_random(128, 2, 1, 1, 1, seed=5)
    args = _inputs(wl, wl.obj, measurements(wl), dev)
    p = _lib.PtychoParams(M=128, S=400, H=wl.H, W=wl.W, N=1, lambda_A=0.0251, dz_A=2.0, pixel_A=0.1)
    loss = torch.zeros((), dtype=torch.float64, device=dev)
    rc = lib.ptycho_loss_grad_noalloc(C.byref(p), args[0].data_ptr(), args[1].data_ptr(), args[2].data_ptr(),
                                      args[3].data_ptr(), loss.data_ptr(), None, None, None)
    assert rc == _lib.PTYCHO_ERR_UNSUPPORTED
