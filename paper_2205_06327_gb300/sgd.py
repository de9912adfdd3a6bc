"""Sequential (mini-batch) gradient descent over the probe positions.

Algorithm 1 updates the reconstruction after every probe location (its inner
loop: per-position gradient, then the update), and also adds each gradient to
an accumulated-gradient buffer; after every T-th location the buffers are
reconciled with the neighbouring tiles and applied as a second update, then
cleared.  On one GPU the data-parallel evaluation is the full-batch gradient
of Eq. 2; this module gives the sequential variant: the positions, in the
caller's (raster) order, are taken in batches of ``batch`` (1 = Algorithm 1's
per-position update, N = full batch), and after each batch O and P are
updated with that batch's gradient (one ``ptycho_step`` call).  With a period
``T`` > 0 each batch is one ``ptycho_step_accumulate`` call instead, which
also adds the batch's object gradient to the buffer and, when the count of
locations reaches a multiple of T, applies the buffer and clears it (the
whole object is one tile here, so reconciling adds nothing).  The buffer
carries over from one epoch to the next, as the paper's loop over locations
runs on without a reset.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from .api import Geometry, Plan, _stream_handle


class SequentialGD:
    def __init__(self, geom: Geometry, batch: int, device, precision: str = "fp32", period: int = 0):
        if batch < 1:
            raise ValueError("batch must be >= 1")
        if period < 0:
            raise ValueError("period must be >= 0")
        self.geom = geom
        self.batch = min(batch, geom.N)
        self.period = period
        self.device = torch.device(device)
        self.acc = (torch.zeros((geom.S, geom.H, geom.W), dtype=torch.complex64, device=self.device)
                    if period else None)
        self.locations = 0  # Algorithm 1's location counter i (runs on across epochs)
        self.plans = {}
        for n in {self.batch, geom.N % self.batch or self.batch}:
            g = Geometry(geom.M, geom.S, geom.H, geom.W, n, geom.lambda_A, geom.dz_A, geom.pixel_A)
            self.plans[n] = Plan(g, self.device, async_check=True, precision=precision)
        self.batch_loss = None

    def epoch(self, pos: torch.Tensor, probe: torch.Tensor, obj: torch.Tensor, meas: torch.Tensor,
              alpha_obj: float, alpha_probe: float) -> torch.Tensor:
        """One pass over all positions; O and P are updated in place after every
        batch.  Returns the loss of every batch, evaluated just before its update
        (float64 device tensor)."""
        N, b = self.geom.N, self.batch
        n_batches = (N + b - 1) // b
        self.batch_loss = torch.zeros(n_batches, dtype=torch.float64, device=self.device)
        stream = _stream_handle(self.device)
        t = C.c_double(0.0)
        for k in range(n_batches):
            i0, i1 = k * b, min(N, (k + 1) * b)
            plan = self.plans[i1 - i0]
            loss_ptr = self.batch_loss.data_ptr() + 8 * k
            if self.period:
                before = self.locations
                self.locations += i1 - i0
                flush = int(self.locations // self.period > before // self.period)
                _lib.check(plan.lib.ptycho_step_accumulate(
                    plan._h, pos[i0:i1].data_ptr(), probe.data_ptr(), obj.data_ptr(), meas[i0:i1].data_ptr(),
                    float(alpha_obj), float(alpha_probe), self.acc.data_ptr(), flush, loss_ptr, stream))
            else:
                _lib.check(plan.lib.ptycho_step(plan._h, pos[i0:i1].data_ptr(), probe.data_ptr(),
                                                obj.data_ptr(), meas[i0:i1].data_ptr(), float(alpha_obj),
                                                float(alpha_probe), 0, loss_ptr, C.byref(t), stream))
        return self.batch_loss

    def close(self):
        for p in self.plans.values():
            p.close()
