"""Plain FP64 CPU oracle for the multislice ptychography loss and gradient.

TEST INFRASTRUCTURE ONLY.  Nothing on the product path may import, call or
execute this module: only the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` use it.  It shares no code with the CUDA path.

What it computes, with the paper's notation (Sec. II-B, Eq. 1; Sec. III, Eq. 2):

* cost F(V) = sum_i sum_k ( |y_i|_k - |G(p, V)_i|_k )^2        (Eq. 1)
  with |y_i| = sqrt(I_i), the measured far-field amplitude;
* G is the multislice model of Sec. II-B: the wave entering slice s is
  multiplied by that slice's transmission, then Fourier transformed,
  propagated, inverse transformed and handed to the next slice; the exit wave
  is Fourier transformed to the detector;
* the image gradient is the sum of the per-position gradients (Eq. 2), each
  non-zero only inside its own probe window (Sec. III).

Readings taken where the paper is silent (all fixed, none are options):

* FFTs are orthonormal, forward kernel exp(-2 pi i ...), data in FFT order
  (DC at [0, 0]); the propagator between slices is the Fresnel kernel
  h(k) = exp(-i pi lambda dz |k|^2), k = fftfreq(M, pixel); S-1 propagations
  separate S slices.
* The unknowns are the complex slice transmissions O_s = exp(i sigma V_s) and
  one probe P shared by all positions; positions are integer top-left corners
  of M x M windows, never wrapped.
* Gradients follow the convention g = dL/dRe + i dL/dIm, so a directional
  derivative along d is Re sum conj(g) d.
* Where |Psi| = 0 the amplitude's subgradient Psi/|Psi| is taken as 0.

Every function evaluates one position at a time and keeps every wave; nothing
is blocked, fused or reordered beyond the definition.
"""
from __future__ import annotations

import numpy as np


# --------------------------------------------------------------------------
# Transforms (Sec. II-B: each slice is Fourier transformed, propagated and
# inverse transformed; the exit wave is Fourier transformed to the detector)
# --------------------------------------------------------------------------

def fft2(x: np.ndarray) -> np.ndarray:
    """Orthonormal 2-D DFT over the last two axes (library primitive)."""
    return np.fft.fft2(x, norm="ortho")


def ifft2(x: np.ndarray) -> np.ndarray:
    """Orthonormal inverse 2-D DFT over the last two axes (library primitive)."""
    return np.fft.ifft2(x, norm="ortho")


def dft2_naive(x: np.ndarray) -> np.ndarray:
    """Orthonormal 2-D DFT written as the double sum, O(M^4); tiny sizes only."""
    My, Mx = x.shape
    out = np.zeros((My, Mx), dtype=np.complex128)
    for ky in range(My):
        for kx in range(Mx):
            acc = 0.0 + 0.0j
            for ny in range(My):
                for nx in range(Mx):
                    acc += x[ny, nx] * np.exp(-2j * np.pi * (ky * ny / My + kx * nx / Mx))
            out[ky, kx] = acc
    return out / np.sqrt(My * Mx)


def fresnel_propagator(M: int, lambda_A: float, dz_A: float, pixel_A: float) -> np.ndarray:
    """Fresnel transfer function h(ky, kx) = exp(-i pi lambda dz (kx^2 + ky^2)).

    k = fftfreq(M, d=pixel) in 1/Angstrom, FFT order; no band limit.
    """
    k = np.fft.fftfreq(M, d=pixel_A)
    k2 = k[:, None] ** 2 + k[None, :] ** 2
    return np.exp(-1j * np.pi * lambda_A * dz_A * k2)


def propagate(x: np.ndarray, h: np.ndarray) -> np.ndarray:
    """Free-space step between slices: inverse FT of h times the FT of x."""
    return ifft2(h * fft2(x))


def window(obj_s: np.ndarray, r, M: int) -> np.ndarray:
    """The M x M patch of one slice at top-left corner r = (y, x)."""
    y, x = int(r[0]), int(r[1])
    return obj_s[y:y + M, x:x + M]


def check_positions(pos: np.ndarray, M: int, H: int, W: int) -> None:
    if pos.ndim != 2 or pos.shape[1] != 2:
        raise ValueError("positions must be [N, 2] (y, x)")
    if len(pos) and (pos.min() < 0 or pos[:, 0].max() > H - M or pos[:, 1].max() > W - M):
        raise ValueError("position window outside the object")


# --------------------------------------------------------------------------
# Forward model G (Sec. II-B) and cost (Eq. 1)
# --------------------------------------------------------------------------

def multislice_waves(probe, obj, r, h):
    """Multislice model G for one position (Sec. II-B).

    Returns (psi, phi, Psi): psi[s] is the wave entering slice s (psi[0] = P),
    phi[s] = psi[s] * O_s[window], and Psi = F phi[S-1] is the far field.
    """
    S = obj.shape[0]
    M = probe.shape[0]
    psi, phi = [], []
    cur = probe.astype(np.complex128)
    for s in range(S):
        psi.append(cur)
        ph = cur * window(obj[s], r, M)
        phi.append(ph)
        if s < S - 1:
            cur = propagate(ph, h)
    Psi = fft2(phi[-1])
    return psi, phi, Psi


def forward(probe, obj, pos, h) -> np.ndarray:
    """Far-field waves G(p, V) for every position, complex128 [N, M, M]."""
    M = probe.shape[0]
    check_positions(pos, M, obj.shape[1], obj.shape[2])
    out = np.empty((len(pos), M, M), dtype=np.complex128)
    for i, r in enumerate(pos):
        out[i] = multislice_waves(probe, obj, r, h)[2]
    return out


def intensities(probe, obj, pos, h) -> np.ndarray:
    """Noise-free measurements |G(p, V)|^2, float64 [N, M, M] (FFT order)."""
    return np.abs(forward(probe, obj, pos, h)) ** 2


def position_loss(Psi, I) -> float:
    """f_i = sum_k (|y_i| - |G_i|)^2 with |y_i| = sqrt(I_i) (Sec. III, f_i)."""
    return float(np.sum((np.abs(Psi) - np.sqrt(I)) ** 2))


def loss(probe, obj, pos, I, h) -> float:
    """F(V) of Eq. 1: the sum of the per-position costs."""
    Psi = forward(probe, obj, pos, h)
    return float(sum(position_loss(Psi[i], I[i]) for i in range(len(pos))))


# --------------------------------------------------------------------------
# Gradient (Eq. 2: sum of per-position gradients, each supported on its window)
# --------------------------------------------------------------------------

def amplitude_residual_grad(Psi, I):
    """g_Psi = 2 (|Psi| - sqrt(I)) Psi/|Psi|, with Psi/|Psi| := 0 where |Psi| = 0."""
    a = np.abs(Psi)
    unit = np.zeros_like(Psi)
    nz = a > 0
    unit[nz] = Psi[nz] / a[nz]
    return 2.0 * (a - np.sqrt(I)) * unit


def position_loss_grad(probe, obj, r, I, h):
    """(f_i, g_O restricted to window i as [S, M, M], g_P) for one position.

    The adjoint runs the forward chain backwards: the far-field transform's
    adjoint is its inverse (orthonormal), the adjoint of multiplying by h is
    multiplying by conj(h), and the transmission phi = psi * O splits the
    incoming gradient into conj(psi) g (object) and conj(O) g (wave).
    """
    S = obj.shape[0]
    M = probe.shape[0]
    psi, phi, Psi = multislice_waves(probe, obj, r, h)
    f = position_loss(Psi, I)
    g_phi = ifft2(amplitude_residual_grad(Psi, I))
    gO = np.zeros((S, M, M), dtype=np.complex128)
    g_psi = None
    for s in range(S - 1, -1, -1):
        gO[s] = np.conj(psi[s]) * g_phi
        g_psi = np.conj(window(obj[s], r, M)) * g_phi
        if s > 0:
            g_phi = ifft2(np.conj(h) * fft2(g_psi))
    return f, gO, g_psi


def loss_grad(probe, obj, pos, I, h):
    """(F, dF/dO, dF/dP): Eq. 1 and the position sum of Eq. 2.

    dF/dO has the shape of the object [S, H, W]; each position adds its
    window-supported gradient at its own window (Sec. III locality).
    """
    M = probe.shape[0]
    check_positions(pos, M, obj.shape[1], obj.shape[2])
    total = 0.0
    gO = np.zeros(obj.shape, dtype=np.complex128)
    gP = np.zeros(probe.shape, dtype=np.complex128)
    for i, r in enumerate(pos):
        f, gO_i, gP_i = position_loss_grad(probe, obj, r, I[i], h)
        total += f
        y, x = int(r[0]), int(r[1])
        gO[:, y:y + M, x:x + M] += gO_i
        gP += gP_i
    return total, gO, gP


def potential_grad(obj, gO, sigma: float = 1.0):
    """dF/dV for O = exp(i sigma V) with V real: sigma * Im(conj(O) * g_O)."""
    return sigma * np.imag(np.conj(obj) * gO)


# --------------------------------------------------------------------------
# Gradient-descent step (Sec. II-B; Algorithm 1's update V <- V - alpha dF/dV,
# taken here at full batch, i.e. on the position sum of Eq. 2)
# --------------------------------------------------------------------------

def step(probe, obj, pos, I, h, alpha_obj: float, alpha_probe: float,
         line_search: bool = False, c: float = 1e-4, max_halvings: int = 20):
    """One full-batch gradient-descent step.  Returns (new_probe, new_obj, F_before, alpha_scale).

    Without line search: O <- O - alpha_obj g_O, P <- P - alpha_probe g_P.
    With Armijo backtracking the pair of step sizes is scaled by t = 1, 1/2,
    1/4, ... (at most ``max_halvings`` halvings) until
        F(x - t a g) <= F(x) - c t (alpha_obj |g_O|^2 + alpha_probe |g_P|^2);
    if no t passes, t = 0 (no update).
    """
    F0, gO, gP = loss_grad(probe, obj, pos, I, h)
    t = 1.0
    if line_search:
        decrease = alpha_obj * np.sum(np.abs(gO) ** 2) + alpha_probe * np.sum(np.abs(gP) ** 2)
        for _ in range(max_halvings + 1):
            Pn = probe - t * alpha_probe * gP
            On = obj - t * alpha_obj * gO
            if loss(Pn, On, pos, I, h) <= F0 - c * t * decrease:
                return Pn, On, F0, t
            t *= 0.5
        return probe.copy(), obj.copy(), F0, 0.0
    return probe - alpha_probe * gP, obj - alpha_obj * gO, F0, t
