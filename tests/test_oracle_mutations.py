"""Planted mistakes in the oracle must fail its pins.

Each case patches one plausible slip into a copy of the oracle's per-position
gradient, multislice model or step (CPU only) and checks that a pin rejects
it: the finite-difference pin for slips in the adjoint, the dense-matrix
multislice pin for slips in the order of the forward model (which the
finite-difference pin cannot see: a wrong forward model with its own exact
adjoint is still self-consistent), and the brute-force Armijo pin for slips
in the line search.
"""
import numpy as np
import pytest

import test_oracle_pins as pins
from oracle import ptycho_oracle as orc
from paper_2205_06327_gb300 import synth


def _problem():
    g = synth.rng(21)
    M, S, H, W = 8, 3, 12, 15
    probe = g.standard_normal((M, M)) + 1j * g.standard_normal((M, M))
    obj = np.exp(1j * g.uniform(-0.6, 0.6, (S, H, W))) * (1 + 0.3 * g.uniform(-1, 1, (S, H, W)))
    pos = np.array([[0, 1], [3, 5], [4, 2], [1, 7]], np.int32)
    h = orc.fresnel_propagator(M, 0.0251, 2.0, 0.1)
    I = orc.intensities(probe, obj, pos, h) * g.uniform(0.5, 1.5, (4, M, M))
    return probe, obj, pos, I, h


def _fd_mismatch(grad_fn):
    probe, obj, pos, I, h = _problem()
    M = probe.shape[0]
    gO = np.zeros(obj.shape, complex)
    gP = np.zeros(probe.shape, complex)
    for i, r in enumerate(pos):
        _, gOi, gPi = grad_fn(probe, obj, r, I[i], h)
        gO[:, r[0]:r[0] + M, r[1]:r[1] + M] += gOi
        gP += gPi
    g = synth.rng(3)
    worst = 0.0
    for _ in range(4):
        dO = g.standard_normal(obj.shape) + 1j * g.standard_normal(obj.shape)
        dP = g.standard_normal(probe.shape) + 1j * g.standard_normal(probe.shape)
        e = 1e-6
        fd = (orc.loss(probe + e * dP, obj + e * dO, pos, I, h)
              - orc.loss(probe - e * dP, obj - e * dO, pos, I, h)) / (2 * e)
        an = np.real(np.vdot(gO, dO) + np.vdot(gP, dP))
        worst = max(worst, abs(fd - an) / abs(fd))
    return worst


def _variant(adj_h=np.conj, psi_conj=True, obj_conj=True, ifft_far=True, factor=2.0):
    def fn(probe, obj, r, I, h):
        S, M = obj.shape[0], probe.shape[0]
        psi, phi, Psi = orc.multislice_waves(probe, obj, r, h)
        a = np.abs(Psi)
        gPsi = factor * (a - np.sqrt(I)) * Psi / a
        g_phi = orc.ifft2(gPsi) if ifft_far else orc.fft2(gPsi)
        gO = np.zeros((S, M, M), complex)
        for s in range(S - 1, -1, -1):
            gO[s] = (np.conj(psi[s]) if psi_conj else psi[s]) * g_phi
            w = orc.window(obj[s], r, M)
            g_psi = (np.conj(w) if obj_conj else w) * g_phi
            if s > 0:
                g_phi = orc.ifft2(adj_h(h) * orc.fft2(g_psi))
        return 0.0, gO, g_psi
    return fn


def test_correct_variant_passes():
    assert _fd_mismatch(_variant()) < 1e-7
    assert _fd_mismatch(orc.position_loss_grad) < 1e-7


@pytest.mark.parametrize("kw", [
    dict(adj_h=lambda h: h),          # propagator not conjugated in the adjoint
    dict(psi_conj=False),             # object gradient without conj(psi)
    dict(obj_conj=False),             # wave gradient without conj(O)
    dict(ifft_far=False),             # far-field adjoint taken as the forward FFT
    dict(factor=1.0),                 # halved gradient (dL/dz-bar instead of dL/dRe + i dL/dIm)
])
def test_planted_mistake_is_caught(kw):
    assert _fd_mismatch(_variant(**kw)) > 1e-3


# ------------------------------------------------- order of the forward model

def _slices_reversed(probe, obj, r, h):
    """Slip: the slices applied last-to-first."""
    return _ordered(probe, obj[::-1], r, h, prop_first=False)


def _propagate_before_transmit(probe, obj, r, h):
    """Slip: every slice propagates the incoming wave before its transmission
    (phi_s = prop(psi_s) O_s), instead of transmitting and then propagating."""
    return _ordered(probe, obj, r, h, prop_first=True)


def _ordered(probe, obj, r, h, prop_first):
    S, M = obj.shape[0], probe.shape[0]
    psi, phi = [], []
    cur = probe.astype(np.complex128)
    for s in range(S):
        if prop_first:
            cur = orc.propagate(cur, h)
        psi.append(cur)
        ph = cur * orc.window(obj[s], r, M)
        phi.append(ph)
        if not prop_first and s < S - 1:
            cur = orc.propagate(ph, h)
        elif prop_first:
            cur = ph
    return psi, phi, orc.fft2(phi[-1])


def test_correct_order_passes_dense_pin():
    pins.check_against_dense(*pins._multislice_problem(3, 43))


@pytest.mark.parametrize("slip", [_slices_reversed, _propagate_before_transmit])
def test_planted_order_mistake_is_caught_by_dense_pin(monkeypatch, slip):
    monkeypatch.setattr(orc, "multislice_waves", slip)
    with pytest.raises(AssertionError):
        pins.check_against_dense(*pins._multislice_problem(3, 43))


# ------------------------------------------------------------- line search

def _armijo_variant(accept_first_halving=False, drop_alpha=False):
    def step(probe, obj, pos, I, h, alpha_obj, alpha_probe, line_search=False, c=1e-4, max_halvings=20):
        F0, gO, gP = orc.loss_grad(probe, obj, pos, I, h)
        na = 1.0 if drop_alpha else alpha_obj
        npb = 1.0 if drop_alpha else alpha_probe
        decrease = na * np.sum(np.abs(gO) ** 2) + npb * np.sum(np.abs(gP) ** 2)
        t = 1.0
        for k in range(max_halvings + 1):
            Pn, On = probe - t * alpha_probe * gP, obj - t * alpha_obj * gO
            if orc.loss(Pn, On, pos, I, h) <= F0 - c * t * decrease or (accept_first_halving and k == 1):
                return Pn, On, F0, t
            t *= 0.5
        return probe.copy(), obj.copy(), F0, 0.0
    return step


def test_correct_armijo_variant_passes():
    for case in pins.ARMIJO_CASES:
        pins.check_armijo(_armijo_variant(), *case)


@pytest.mark.parametrize("kw", [dict(accept_first_halving=True), dict(drop_alpha=True)])
def test_planted_armijo_mistake_is_caught(kw):
    failed = 0
    for case in pins.ARMIJO_CASES:
        try:
            pins.check_armijo(_armijo_variant(**kw), *case)
        except AssertionError:
            failed += 1
    assert failed >= 1
