"""Several independent reconstructions advanced together, one CUDA graph per iteration.

Each problem keeps its own plan (tables, workspace), device tensors and
shape; one gradient-descent iteration of all problems -- for every problem the
loss, both gradients (Eq. 1, Eq. 2) and the in-place update of O and P -- is
one library call (ptycho_multi_step), captured once in a CUDA graph and
replayed, so an iteration costs one graph launch however many problems and
kernels it contains.  The workspace budget
is shared: each plan gets ``workspace_bytes / n_problems`` and chunks its
positions to fit.

Windows: 64 and 128 run the register-resident kernels; any other M = 2^a 3^b
in [8, 4096] runs the generic batched-FFT path (FP32 only); the tensor-core
precisions take M = 128.  ``supported(M)`` says which.
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import _lib
from .api import Geometry, Plan, _stream_handle

def _smooth(M: int) -> bool:
    m = M
    for p in (2, 3):
        while m % p == 0:
            m //= p
    return m == 1


def supported(M: int, precision: str = "fp32") -> bool:
    if precision == "fp32":
        return 8 <= M <= 4096 and _smooth(M)
    return M == 128


@dataclass
class Problem:
    geom: Geometry
    pos: torch.Tensor     # int32 [N, 2] on the device
    probe: torch.Tensor   # complex64 [M, M], updated in place
    obj: torch.Tensor     # complex64 [S, H, W], updated in place
    meas: torch.Tensor    # float32 [N, M, M]
    tile: tuple[int, int] = (0, 0)


class MultiProblem:
    def __init__(self, problems: list[Problem], device, precision: str = "fp32",
                 workspace_bytes: int = 96 << 30):
        for p in problems:
            if not supported(p.geom.M, precision):
                raise ValueError(f"window {p.geom.M} is not supported with precision {precision}")
        self.device = torch.device(device)
        self.problems = problems
        per = max(workspace_bytes // max(len(problems), 1), 1 << 20)
        self.plans = [Plan(p.geom, self.device, workspace_bytes=per, tile=p.tile, async_check=True,
                           precision=precision) for p in problems]
        self.loss = torch.zeros(len(problems), dtype=torch.float64, device=self.device)
        self.graph = None
        self._alphas = None

    @property
    def positions_per_iteration(self) -> int:
        return sum(p.geom.N for p in self.problems)

    def _entries(self, grads=None):
        arr = (_lib.PtychoProblem * len(self.problems))()
        for i, (p, plan) in enumerate(zip(self.problems, self.plans)):
            e = arr[i]
            e.plan = plan._h.value
            e.pos_yx, e.probe, e.obj, e.meas_I = (p.pos.data_ptr(), p.probe.data_ptr(), p.obj.data_ptr(),
                                                  p.meas.data_ptr())
            e.loss_out = self.loss.data_ptr() + 8 * i
            if grads is not None:
                e.grad_obj, e.grad_probe = grads[i][0].data_ptr(), grads[i][1].data_ptr()
        return arr

    def step_all(self, alpha_obj: float, alpha_probe: float) -> None:
        """One fixed-step gradient-descent iteration of every problem: one library call."""
        arr = self._entries()
        with torch.cuda.device(self.device):
            _lib.check(self.plans[0].lib.ptycho_multi_step(arr, len(self.problems), float(alpha_obj),
                                                           float(alpha_probe), _stream_handle(self.device)))

    def loss_grad_all(self):
        """(F, dF/dO, dF/dP) of every problem (F in self.loss), one library call."""
        grads = [(torch.empty_like(p.obj), torch.empty_like(p.probe)) for p in self.problems]
        arr = self._entries(grads)
        with torch.cuda.device(self.device):
            _lib.check(self.plans[0].lib.ptycho_multi_loss_grad(arr, len(self.problems),
                                                                _stream_handle(self.device)))
        return self.loss, grads

    def capture(self, alpha_obj: float, alpha_probe: float, warmup: int = 1) -> None:
        """Capture one iteration of all problems in a CUDA graph (after eager warm-up
        iterations, which also allocate every workspace before capture)."""
        side = torch.cuda.Stream(self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            for _ in range(warmup):
                self.step_all(alpha_obj, alpha_probe)
        torch.cuda.current_stream(self.device).wait_stream(side)
        torch.cuda.synchronize(self.device)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, capture_error_mode="relaxed"):
            self.step_all(alpha_obj, alpha_probe)
        self.graph = g
        self._alphas = (alpha_obj, alpha_probe)

    def run(self, iterations: int) -> torch.Tensor:
        """Replay the captured iteration; returns the loss of every problem before
        the last iteration (float64 device tensor)."""
        if self.graph is None:
            raise RuntimeError("capture() first")
        for _ in range(iterations):
            self.graph.replay()
        return self.loss

    def check_status(self) -> None:
        for plan in self.plans:
            plan.status()

    def close(self) -> None:
        self.graph = None
        for plan in self.plans:
            plan.close()
