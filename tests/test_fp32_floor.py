"""The rounding floor of plain FP32 on long slice chains (CPU, no GPU).

A single-precision evaluation of the same chain (SciPy FFTs, complex64
pointwise arithmetic) against the FP64 oracle on the 16-slice workload: its
gradient error grows with the number of slices and, near the noisy optimum,
exceeds 1e-5 -- the FP32 arithmetic itself, not a kernel, sets that floor.
The GPU parity tests hold the CUDA path to 1.5x this model's error there.
"""
import numpy as np

from oracle import ptycho_oracle as orc
from paper_2205_06327_gb300 import synth
from tests.helpers import c64, fp32_chain_loss_grad, measurements, propagator, rel_l2


def _errors(S):
    wl = synth.workload_multislice()
    wl.obj, wl.S = wl.obj[:S], S
    wl.pos = wl.pos.reshape(24, 24, 2)[8:12, 8:12].reshape(-1, 2).copy()
    I = measurements(wl, counts_seed=1002)
    h = propagator(wl)
    L, gO, gP = orc.loss_grad(c64(wl.probe), c64(wl.obj), wl.pos, I.astype(np.float64), h)
    l, go, gp = fp32_chain_loss_grad(wl.probe, wl.obj, wl.pos, I, h)
    return abs(l - L) / L, rel_l2(go, gO), rel_l2(gp, gP)


def test_fp32_gradient_floor_grows_with_slices():
    e1 = _errors(1)
    e16 = _errors(16)
    assert max(e1) < 1e-5                  # one slice: plain FP32 is well inside 1e-5
    assert e16[0] < 1e-5                   # the loss stays inside 1e-5
    assert max(e16[1:]) > 3 * max(e1[1:])  # the gradient error grows with the chain
    assert max(e16[1:]) > 5e-6             # and reaches the 1e-5 scale at 16 slices, at the optimum
