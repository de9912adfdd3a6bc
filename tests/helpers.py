"""Shared helpers for the GPU parity tests (inputs from synth, expectations from the oracle)."""
from __future__ import annotations

import numpy as np

from oracle import ptycho_oracle as orc
from paper_2205_06327_gb300 import synth

TOL_FP32 = 1e-5   # rel-L2 bound of the FP32 path against the FP64 oracle


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def propagator(wl):
    return orc.fresnel_propagator(wl.M, wl.lambda_A, wl.dz_A, wl.pixel_A)


def measurements(wl, counts_seed=None, scale=1.0):
    """float32 intensities from the oracle's forward model at the true object."""
    I = orc.intensities(wl.probe, wl.obj, wl.pos, propagator(wl)) * scale
    if wl.counts is not None and counts_seed is not None:
        return synth.poisson_counts(I, counts_seed)
    return I.astype(np.float32)


def start_object(wl, kind: str, seed: int = 0):
    """Evaluation points: 'truth', 'vacuum' (O = 1) or 'perturbed' truth."""
    if kind == "truth":
        return wl.obj.copy()
    if kind == "vacuum":
        return np.ones_like(wl.obj)
    g = synth.rng(seed + 99)
    return wl.obj * np.exp(0.1j * g.standard_normal(wl.obj.shape)) * (1 + 0.05 * g.uniform(-1, 1, wl.obj.shape))


def to_dev(a, dtype, device):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).to(device)
