"""The host-buffer entry point (ptycho_loss_grad_host): the same results as the
device-pointer call, bit for bit, while the intensities of all but the first
chain wave are uploaded beside the kernels; host-side position checks and
argument errors."""
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


def _case(M, S, ny, nx, step, seed):
    wl = synth.workload_random(M, S, ny, nx, step, seed=seed, amp_jitter=0.1)
    I = (measurements(wl) * 1.2).astype(np.float32)
    return wl, start_object(wl, "perturbed", seed), I


def _host(a, dtype, pinned):
    t = torch.from_numpy(np.ascontiguousarray(a)).to(dtype)
    return t.pin_memory() if pinned else t


def _compare(dev, wl, obj, I, pinned=True, pageable_out=False, **plan_kw):
    """Host entry vs device entry on one plan each; returns the host results
    (outputs in pinned host tensors, or in caller-given pageable ones)."""
    from paper_2205_06327_gb300 import api
    g = api.Geometry(wl.M, wl.S, wl.H, wl.W, wl.N, wl.lambda_A, wl.dz_A, wl.pixel_A)
    ph = api.Plan(g, dev, **plan_kw)
    pd = api.Plan(g, dev, **plan_kw)
    outs = {}
    if pageable_out:
        outs = dict(out_obj=torch.empty((wl.S, wl.H, wl.W), dtype=torch.complex64),
                    out_probe=torch.empty((wl.M, wl.M), dtype=torch.complex64))
    hl, hO, hP = ph.loss_grad(_host(wl.pos, torch.int32, pinned), _host(wl.probe, torch.complex64, pinned),
                              _host(obj, torch.complex64, pinned), _host(I, torch.float32, pinned), **outs)
    assert not hO.is_cuda and not hP.is_cuda and not hl.is_cuda
    dl, dO, dP = pd.loss_grad(to_dev(wl.pos, torch.int32, dev), to_dev(wl.probe, torch.complex64, dev),
                              to_dev(obj, torch.complex64, dev), to_dev(I, torch.float32, dev))
    torch.cuda.synchronize()
    assert float(hl) == float(dl)
    assert torch.equal(hO, dO.cpu()) and torch.equal(hP, dP.cpu())
    chunk = ph.chunk
    ph.close()
    pd.close()
    return hl, hO, hP, chunk


def test_host_entry_split_waves_matches_device_and_oracle(dev):
    # 192 positions at M = 128: the first chain wave, then the rest after the
    # second upload (and a partial last wave beside the accumulation)
    wl, obj, I = _case(128, 2, 16, 12, 8, 901)
    assert wl.N > torch.cuda.get_device_properties(dev).multi_processor_count
    hl, hO, hP, _ = _compare(dev, wl, obj, I)
    L, gO, gP = orc.loss_grad(c64(wl.probe), c64(obj), wl.pos, I.astype(np.float64), propagator(wl))
    assert abs(float(hl) - L) <= 1e-5 * abs(L)
    assert rel_l2(hO.numpy(), gO) <= 1e-5 and rel_l2(hP.numpy(), gP) <= 1e-5


def test_host_entry_pageable_inputs(dev):
    wl, obj, I = _case(128, 2, 14, 12, 9, 902)
    _compare(dev, wl, obj, I, pinned=False)
    _compare(dev, wl, obj, I, pinned=False, pageable_out=True)
    _compare(dev, wl, obj, I, pinned=True, pageable_out=True)


def test_host_entry_several_chunks(dev):
    # a workspace of one wave per chunk: the split applies to the first chunk only
    wl, obj, I = _case(128, 2, 20, 18, 6, 903)
    per_pos = (1 + 2 + 1) * 128 * 128 * 8 + 8
    _, _, _, chunk = _compare(dev, wl, obj, I, workspace_bytes=160 * per_pos)
    assert chunk < wl.N


def test_host_entry_small_window_and_recompute(dev):
    wl, obj, I = _case(64, 5, 26, 28, 4, 904)  # 728 positions: more than one wave at M = 64
    _compare(dev, wl, obj, I)
    _compare(dev, wl, obj, I, ckpt_every=2)


def test_host_entry_generic_window_and_split_precision(dev):
    wl, obj, I = _case(96, 2, 3, 4, 11, 905)
    _compare(dev, wl, obj, I)
    wl, obj, I = _case(128, 2, 13, 13, 9, 906)
    _compare(dev, wl, obj, I, precision="fp16x3")


def test_host_entry_reuses_buffers_across_calls(dev):
    from paper_2205_06327_gb300 import api
    wl, obj, I = _case(128, 2, 14, 12, 8, 907)
    g = api.Geometry(wl.M, wl.S, wl.H, wl.W, wl.N, wl.lambda_A, wl.dz_A, wl.pixel_A)
    ph, pd = api.Plan(g, dev), api.Plan(g, dev)
    pos_h = _host(wl.pos, torch.int32, True)
    for k in range(3):  # new object and intensities on every call
        o = start_object(wl, "perturbed", 50 + k)
        Ik = (I * (1.0 + 0.1 * k)).astype(np.float32)
        hl, hO, hP = ph.loss_grad(pos_h, _host(wl.probe, torch.complex64, True), _host(o, torch.complex64, True),
                                  _host(Ik, torch.float32, True))
        dl, dO, dP = pd.loss_grad(to_dev(wl.pos, torch.int32, dev), to_dev(wl.probe, torch.complex64, dev),
                                  to_dev(o, torch.complex64, dev), to_dev(Ik, torch.float32, dev))
        torch.cuda.synchronize()
        assert float(hl) == float(dl) and torch.equal(hO, dO.cpu()) and torch.equal(hP, dP.cpu())
    # gradients not asked for: loss only, same value
    hl2, hO2, hP2 = ph.loss_grad(pos_h, _host(wl.probe, torch.complex64, True), _host(o, torch.complex64, True),
                                 _host(Ik, torch.float32, True), want_obj=False, want_probe=False)
    assert hO2 is None and hP2 is None and float(hl2) == float(hl)
    ph.close()
    pd.close()


def test_host_entry_errors(dev):
    import ctypes as C
    from paper_2205_06327_gb300 import _lib, api
    from paper_2205_06327_gb300._lib import PtychoError
    wl, obj, I = _case(64, 1, 3, 3, 10, 908)
    g = api.Geometry(wl.M, wl.S, wl.H, wl.W, wl.N, wl.lambda_A, wl.dz_A, wl.pixel_A)
    plan = api.Plan(g, dev)
    pos, probe = _host(wl.pos, torch.int32, True), _host(wl.probe, torch.complex64, True)
    o, Ih = _host(obj, torch.complex64, True), _host(I, torch.float32, True)
    bad = pos.clone()
    bad[4, 1] = wl.W - wl.M + 1  # window past the right edge: caught on the host, nothing launched
    with pytest.raises(PtychoError, match="position 4"):
        plan.loss_grad(bad, probe, o, Ih)
    lib = _lib.load()
    loss = C.c_double(0.0)
    with torch.cuda.device(dev):
        stream = torch.cuda.current_stream(dev).cuda_stream
        probe_d = probe.to(dev)  # a device array where a host one belongs
        rc = lib.ptycho_loss_grad_host(plan._h, pos.data_ptr(), probe_d.data_ptr(), o.data_ptr(), Ih.data_ptr(),
                                       C.addressof(loss), None, None, stream)
        assert rc == _lib.PTYCHO_ERR_ARG and b"host pointer" in lib.ptycho_last_error()
        rc = lib.ptycho_loss_grad_host(plan._h, pos.data_ptr(), probe.data_ptr(), o.data_ptr(), Ih.data_ptr(),
                                       None, None, None, stream)
        assert rc == _lib.PTYCHO_ERR_ARG and b"loss_out" in lib.ptycho_last_error()
    # the plan still works after the refused calls
    l1, _, _ = plan.loss_grad(pos, probe, o, Ih)
    L = orc.loss(c64(wl.probe), c64(obj), wl.pos, I.astype(np.float64), propagator(wl))
    assert abs(float(l1) - L) <= 1e-5 * abs(L)
    plan.close()


def test_host_entry_no_positions(dev):
    from paper_2205_06327_gb300 import api
    wl, obj, _ = _case(64, 2, 2, 2, 10, 909)
    g = api.Geometry(wl.M, wl.S, wl.H, wl.W, 0, wl.lambda_A, wl.dz_A, wl.pixel_A)
    plan = api.Plan(g, dev)
    l0, gO, gP = plan.loss_grad(torch.zeros((0, 2), dtype=torch.int32), _host(wl.probe, torch.complex64, True),
                                _host(obj, torch.complex64, True), torch.zeros((0, 64, 64), dtype=torch.float32))
    assert float(l0) == 0.0 and not gO.abs().any() and not gP.abs().any()
    plan.close()


def test_host_entry_reports_a_device_timeout(dev):
    """The synchronous host-buffer call reads the device error word itself:
    the split-product kernel's self-test wait (no MMAs issued, the bounded
    wait expires after about 1 s) comes back as PTYCHO_ERR_TIMEOUT from the
    call, the word is cleared, and the next plain evaluation is correct."""
    import ctypes as C

    from paper_2205_06327_gb300 import _lib
    wl, obj, I = _case(128, 2, 1, 1, 9, 910)
    lib = _lib.load()
    p = _lib.PtychoParams(M=wl.M, S=wl.S, H=wl.H, W=wl.W, N=wl.N, lambda_A=wl.lambda_A, dz_A=wl.dz_A,
                          pixel_A=wl.pixel_A, precision=_lib.PTYCHO_FP16X3,
                          flags=_lib.PTYCHO_FLAG_SELFTEST_TIMEOUT)
    h = C.c_void_p()
    assert lib.ptycho_plan_create(C.byref(h), C.byref(p)) == _lib.PTYCHO_OK
    pos, probe = _host(wl.pos, torch.int32, True), _host(wl.probe, torch.complex64, True)
    o, Ih = _host(obj, torch.complex64, True), _host(I, torch.float32, True)
    loss = C.c_double(0.0)
    with torch.cuda.device(dev):
        rc = lib.ptycho_loss_grad_host(h, pos.data_ptr(), probe.data_ptr(), o.data_ptr(), Ih.data_ptr(),
                                       C.addressof(loss), None, None, torch.cuda.current_stream(dev).cuda_stream)
    assert rc == _lib.PTYCHO_ERR_TIMEOUT and b"gave up" in lib.ptycho_last_error()
    assert lib.ptycho_plan_status(h) == _lib.PTYCHO_OK  # cleared by the call
    assert lib.ptycho_plan_destroy(h) == _lib.PTYCHO_OK
    _compare(dev, wl, obj, I, precision="fp16x3")
