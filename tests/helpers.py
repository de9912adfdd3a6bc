"""Shared helpers for the GPU parity tests (inputs from synth, expectations from the oracle)."""
from __future__ import annotations

import numpy as np

from oracle import ptycho_oracle as orc
from paper_2205_06327_gb300 import synth

TOL_FP32 = 1e-5   # rel-L2 bound of the FP32 path against the FP64 oracle


def c64(a):
    """The complex64 values the GPU path receives, as complex128 for the oracle."""
    return np.asarray(a).astype(np.complex64).astype(np.complex128)


def fp32_chain_loss_grad(probe, obj, pos, I, h):
    """The same chain evaluated with single-precision FFTs (SciPy) and complex64
    pointwise arithmetic: an error model of plain FP32, not a reference value.
    Used to state the rounding floor that FP32 arithmetic itself reaches."""
    import scipy.fft as sf
    M, S = probe.shape[0], obj.shape[0]
    P, O, h32 = probe.astype(np.complex64), obj.astype(np.complex64), h.astype(np.complex64)
    f = lambda x: sf.fft2(x, norm="ortho")
    fi = lambda x: sf.ifft2(x, norm="ortho")
    gO = np.zeros(obj.shape, np.complex64)
    gP = np.zeros(probe.shape, np.complex64)
    L = 0.0
    for i, (y, x) in enumerate(pos):
        psi, cur = [], P
        for s in range(S):
            psi.append(cur)
            ph = cur * O[s, y:y + M, x:x + M]
            if s < S - 1:
                cur = fi(h32 * f(ph))
        Psi = f(ph)
        a = np.abs(Psi)
        d = a - np.sqrt(I[i].astype(np.float32))
        L += float(np.sum(d.astype(np.float64) ** 2))
        g = np.where(a > 0, 2 * d * Psi / np.where(a > 0, a, 1), 0).astype(np.complex64)
        gphi = fi(g)
        for s in range(S - 1, -1, -1):
            gO[s, y:y + M, x:x + M] += np.conj(psi[s]) * gphi
            gpsi = np.conj(O[s, y:y + M, x:x + M]) * gphi
            if s > 0:
                gphi = fi(np.conj(h32) * f(gpsi))
        gP += gpsi
    return L, gO, gP


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


# ------------------------------------------------------------------ process-pool oracle pieces
# Workers of a spawn pool rebuild the seeded workload themselves (the inputs
# are deterministic), so only positions, detector frames and small results
# cross the process boundary.

_POOL_STATE: dict = {}


def pool_init(workload_fn: str, start_kind: str, start_seed: int) -> None:
    wl = getattr(synth, workload_fn)()
    _POOL_STATE["wl"] = wl
    _POOL_STATE["probe"] = c64(wl.probe)
    _POOL_STATE["truth"] = c64(wl.obj)
    _POOL_STATE["start"] = c64(start_object(wl, start_kind, start_seed))
    _POOL_STATE["h"] = propagator(wl)


def pool_intensities(idx):
    """Oracle intensities |G|^2 at the true object for positions idx (float64)."""
    st = _POOL_STATE
    return orc.intensities(st["probe"], st["truth"], st["wl"].pos[idx], st["h"])


def pool_region_grad(args):
    """One position's dF/dO (oracle, FP64) and the FP32 error model's, both
    restricted to slices `ss` and the pixel block [y0, y1) x [x0, x1)."""
    i, I_i, ss, y0, y1, x0, x1 = args
    st = _POOL_STATE
    wl, M = st["wl"], st["wl"].M
    r = wl.pos[i]
    _, gO_i, _ = orc.position_loss_grad(st["probe"], st["start"], r, I_i.astype(np.float64), st["h"])
    _, f32, _ = fp32_chain_loss_grad(st["probe"], st["start"][:, r[0]:r[0] + M, r[1]:r[1] + M],
                                     np.array([[0, 0]]), I_i[None], st["h"])
    out = np.zeros((2, len(ss), y1 - y0, x1 - x0), np.complex128)
    ya, yb = max(y0, r[0]), min(y1, r[0] + M)
    xa, xb = max(x0, r[1]), min(x1, r[1] + M)
    if ya < yb and xa < xb:
        out[0, :, ya - y0:yb - y0, xa - x0:xb - x0] = gO_i[ss][:, ya - r[0]:yb - r[0], xa - r[1]:xb - r[1]]
        out[1, :, ya - y0:yb - y0, xa - x0:xb - x0] = f32[ss][:, ya - r[0]:yb - r[0], xa - r[1]:xb - r[1]]
    return out
