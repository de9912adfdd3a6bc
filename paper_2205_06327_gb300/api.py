"""PyTorch-facing wrapper of libptycho (the C-ABI in include/ptycho.h).

PyTorch supplies device memory and streams; every step of the computation
runs in the library's CUDA kernels.  Tensors:

* ``pos``   int32  [N, 2] (y, x) top-left window corners
* ``probe`` complex64 [M, M]
* ``obj``   complex64 [S, H, W] slice transmissions
* ``meas``  float32 [N, M, M] measured intensities, FFT order

Host (CPU) tensors are accepted and copied to the plan's device first; the
results then come back to the host as well.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import torch

from . import _lib
from ._lib import PtychoParams, check


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _stream_handle(device: torch.device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


@dataclass
class Geometry:
    M: int
    S: int
    H: int
    W: int
    N: int
    lambda_A: float = 0.0251
    dz_A: float = 2.0
    pixel_A: float = 0.1


class Plan:
    """A ``ptycho_plan``: tables and workspace for one problem shape."""

    def __init__(self, geom: Geometry, device: torch.device | int | str = "cuda",
                 workspace_bytes: int = 0, tile: tuple[int, int] = (0, 0), async_check: bool = False,
                 timing: bool = False, ckpt_every: int | str = 0, precision: str = "fp32"):
        if not torch.cuda.is_available():
            raise RuntimeError("libptycho needs a CUDA device; there is no CPU fallback")
        self.lib = _lib.load()
        self.geom = geom
        self.device = torch.device(device)
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        p = PtychoParams()
        p.M, p.S, p.H, p.W, p.N = geom.M, geom.S, geom.H, geom.W, geom.N
        p.lambda_A, p.dz_A, p.pixel_A = geom.lambda_A, geom.dz_A, geom.pixel_A
        codes = {"fp32": _lib.PTYCHO_FP32, "bf16x3": _lib.PTYCHO_BF16X3, "fp16x3": _lib.PTYCHO_FP16X3}
        if precision not in codes:
            raise ValueError(f"precision must be one of {sorted(codes)}")
        p.precision = codes[precision]
        p.flags = (_lib.PTYCHO_FLAG_ASYNC_CHECK if async_check else 0) | (_lib.PTYCHO_FLAG_TIMING if timing else 0)
        p.workspace_bytes = int(workspace_bytes)
        p.tile_h, p.tile_w = int(tile[0]), int(tile[1])
        p.ckpt_every = _lib.PTYCHO_CKPT_AUTO if ckpt_every == "auto" else int(ckpt_every)
        self._params = p
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib.ptycho_plan_create(C.byref(h), C.byref(p)))
        self._h = h

    # ------------------------------------------------------------------ info
    @property
    def chunk(self) -> int:
        c, w = C.c_int32(), C.c_int64()
        check(self.lib.ptycho_plan_info(self._h, C.byref(c), C.byref(w)))
        return c.value

    @property
    def workspace_bytes(self) -> int:
        c, w = C.c_int32(), C.c_int64()
        check(self.lib.ptycho_plan_info(self._h, C.byref(c), C.byref(w)))
        return w.value

    def timing(self, reset: bool = True) -> dict:
        """Per-kernel-family device milliseconds and launch counts since the last reset."""
        t = _lib.PtychoTiming()
        with torch.cuda.device(self.device):
            check(self.lib.ptycho_plan_timing(self._h, C.byref(t), int(reset)))
        return t.as_dict()

    def status(self) -> None:
        with torch.cuda.device(self.device):
            check(self.lib.ptycho_plan_status(self._h))

    def close(self) -> None:
        if getattr(self, "_h", None) is not None and self._h.value:
            with torch.cuda.device(self.device):
                self.lib.ptycho_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --------------------------------------------------------------- helpers
    def _dev(self, t: torch.Tensor, dtype: torch.dtype, shape: tuple, name: str) -> torch.Tensor:
        if t.dtype != dtype:
            raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
        if t.device != self.device:
            t = t.to(self.device, non_blocking=True)
        return t.contiguous()

    def _to_host(self, *ts):
        """Device results to fresh pinned host tensors: asynchronous copies on the
        current stream (pinned blocks come from torch's host caching allocator),
        then one synchronisation."""
        out = []
        for t in ts:
            if t is None:
                out.append(None)
                continue
            h = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
            h.copy_(t, non_blocking=True)
            out.append(h)
        torch.cuda.current_stream(self.device).synchronize()
        return out

    def _inputs(self, pos, probe, obj, meas=None):
        g = self.geom
        pos = self._dev(pos, torch.int32, (g.N, 2), "pos")
        probe = self._dev(probe, torch.complex64, (g.M, g.M), "probe")
        obj = self._dev(obj, torch.complex64, (g.S, g.H, g.W), "obj")
        if meas is not None:
            meas = self._dev(meas, torch.float32, (g.N, g.M, g.M), "meas")
        return pos, probe, obj, meas

    # ------------------------------------------------------------ operations
    def forward(self, pos, probe, obj, want_psi: bool = True, want_intensity: bool = False):
        """Far fields G(p, V) (Sec. II-B).  Returns (psi or None, intensity or None)."""
        host = not probe.is_cuda
        g = self.geom
        pos, probe, obj, _ = self._inputs(pos, probe, obj)
        psi = torch.empty((g.N, g.M, g.M), dtype=torch.complex64, device=self.device) if want_psi else None
        inten = torch.empty((g.N, g.M, g.M), dtype=torch.float32, device=self.device) if want_intensity else None
        with torch.cuda.device(self.device):
            check(self.lib.ptycho_forward(self._h, _ptr(pos), _ptr(probe), _ptr(obj), _ptr(psi), _ptr(inten),
                                          _stream_handle(self.device)))
        if host:
            with torch.cuda.device(self.device):
                psi, inten = self._to_host(psi, inten)
        return psi, inten

    def loss_grad(self, pos, probe, obj, meas, want_obj: bool = True, want_probe: bool = True,
                  out_obj: torch.Tensor | None = None, out_probe: torch.Tensor | None = None):
        """(F, dF/dO, dF/dP) of Eq. 1 / Eq. 2.  F is a float64 0-d tensor on the device.

        With every input on the host the call goes through ptycho_loss_grad_host
        (uploads overlapped with the chain) and returns host tensors."""
        host = not probe.is_cuda
        g = self.geom
        if all(not t.is_cuda for t in (pos, probe, obj, meas)):
            return self._loss_grad_host(pos, probe, obj, meas, want_obj, want_probe, out_obj, out_probe)
        pos, probe, obj, meas = self._inputs(pos, probe, obj, meas)
        gO = out_obj if out_obj is not None else (
            torch.empty((g.S, g.H, g.W), dtype=torch.complex64, device=self.device) if want_obj else None)
        gP = out_probe if out_probe is not None else (
            torch.empty((g.M, g.M), dtype=torch.complex64, device=self.device) if want_probe else None)
        loss = torch.empty((), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            check(self.lib.ptycho_loss_grad(self._h, _ptr(pos), _ptr(probe), _ptr(obj), _ptr(meas), _ptr(loss),
                                            _ptr(gO), _ptr(gP), _stream_handle(self.device)))
        if host:
            with torch.cuda.device(self.device):
                loss, gO, gP = self._to_host(loss, gO, gP)
        return loss, gO, gP

    def _loss_grad_host(self, pos, probe, obj, meas, want_obj, want_probe, out_obj, out_probe):
        g = self.geom

        def inp(t, dtype, shape, name):
            if t.dtype != dtype:
                raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
            if tuple(t.shape) != tuple(shape):
                raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
            return t.contiguous()

        def out(t, shape, name, want):
            if t is None:
                return torch.empty(shape, dtype=torch.complex64, pin_memory=True) if want else None
            if t.is_cuda or t.dtype != torch.complex64 or tuple(t.shape) != tuple(shape) or not t.is_contiguous():
                raise ValueError(f"{name} must be a contiguous complex64 host tensor of shape {tuple(shape)}")
            return t

        pos = inp(pos, torch.int32, (g.N, 2), "pos")
        probe = inp(probe, torch.complex64, (g.M, g.M), "probe")
        obj = inp(obj, torch.complex64, (g.S, g.H, g.W), "obj")
        meas = inp(meas, torch.float32, (g.N, g.M, g.M), "meas")
        gO = out(out_obj, (g.S, g.H, g.W), "out_obj", want_obj)
        gP = out(out_probe, (g.M, g.M), "out_probe", want_probe)
        loss = torch.empty((), dtype=torch.float64)
        with torch.cuda.device(self.device):
            check(self.lib.ptycho_loss_grad_host(self._h, _ptr(pos), _ptr(probe), _ptr(obj), _ptr(meas),
                                                 _ptr(loss), _ptr(gO), _ptr(gP), _stream_handle(self.device)))
        return loss, gO, gP

    def step(self, pos, probe: torch.Tensor, obj: torch.Tensor, meas, alpha_obj: float, alpha_probe: float,
             line_search: bool = False):
        """One full-batch gradient-descent step, in place on device tensors ``probe`` and ``obj``.

        Returns (F before the step as a float64 device tensor, accepted step scale t)."""
        if not (probe.is_cuda and obj.is_cuda and probe.is_contiguous() and obj.is_contiguous()):
            raise ValueError("step updates probe and obj in place: pass contiguous device tensors")
        pos, _, _, meas = self._inputs(pos, probe, obj, meas)
        loss = torch.empty((), dtype=torch.float64, device=self.device)
        t = C.c_double(0.0)
        with torch.cuda.device(self.device):
            check(self.lib.ptycho_step(self._h, _ptr(pos), _ptr(probe), _ptr(obj), _ptr(meas), float(alpha_obj),
                                       float(alpha_probe), int(bool(line_search)), _ptr(loss), C.byref(t),
                                       _stream_handle(self.device)))
        return loss, t.value


def version() -> str:
    return _lib.load().ptycho_version().decode()


def potential_to_transmission(V: torch.Tensor, sigma: float = 1.0) -> torch.Tensor:
    """O = exp(i sigma V) on the device (V float32, any shape)."""
    if not V.is_cuda or V.dtype != torch.float32:
        raise TypeError("V must be a float32 CUDA tensor")
    V = V.contiguous()
    O = torch.empty(V.shape, dtype=torch.complex64, device=V.device)
    lib = _lib.load()
    with torch.cuda.device(V.device):
        check(lib.ptycho_potential_to_transmission(V.data_ptr(), O.data_ptr(), V.numel(), float(sigma),
                                                   _stream_handle(V.device)))
    return O


def potential_grad(obj: torch.Tensor, grad_obj: torch.Tensor, sigma: float = 1.0) -> torch.Tensor:
    """dF/dV = sigma * Im(conj(O) dF/dO) on the device."""
    if not (obj.is_cuda and grad_obj.is_cuda) or obj.dtype != torch.complex64 or grad_obj.dtype != torch.complex64:
        raise TypeError("obj and grad_obj must be complex64 CUDA tensors")
    if obj.shape != grad_obj.shape:
        raise ValueError("obj and grad_obj must have the same shape")
    obj, grad_obj = obj.contiguous(), grad_obj.contiguous()
    gV = torch.empty(obj.shape, dtype=torch.float32, device=obj.device)
    lib = _lib.load()
    with torch.cuda.device(obj.device):
        check(lib.ptycho_potential_grad(obj.data_ptr(), grad_obj.data_ptr(), gV.data_ptr(), obj.numel(),
                                        float(sigma), _stream_handle(obj.device)))
    return gV
