"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a naive DFT,
Parseval, the closed-form Fresnel propagation of a Gaussian, explicit
Jacobian matrices, central finite differences, invariances of Eq. 1 and the
locality/sum structure of Eq. 2 (Sec. III).  Sizes are tiny so the whole
file runs in seconds on CPU.
"""
import numpy as np
import pytest

import dense_multislice as dm
from oracle import ptycho_oracle as orc
from paper_2205_06327_gb300 import synth

RTOL_FD = 1e-7


def _rand_c(g, shape):
    return g.standard_normal(shape) + 1j * g.standard_normal(shape)


def _small_problem(seed=7, M=8, S=3, H=13, W=15, N=5, noise=True):
    """Non-square object, asymmetric positions, non-unimodular transmissions."""
    g = synth.rng(seed)
    probe = _rand_c(g, (M, M))
    obj = np.exp(1j * g.uniform(-0.5, 0.5, (S, H, W))) * (1 + 0.3 * g.uniform(-1, 1, (S, H, W)))
    pos = np.stack([g.integers(0, H - M + 1, N), g.integers(0, W - M + 1, N)], 1).astype(np.int32)
    h = orc.fresnel_propagator(M, 0.0251, 2.0, 0.1)
    I_true = orc.intensities(probe, obj, pos, h)
    I = I_true * g.uniform(0.5, 1.5, I_true.shape) if noise else I_true
    return probe, obj, pos, I, h


# ---------------------------------------------------------------- transforms

@pytest.mark.parametrize("shape", [(4, 4), (6, 6), (8, 8), (12, 12), (4, 6)])
def test_fft_matches_naive_dft(shape):
    g = synth.rng(1)
    x = _rand_c(g, shape)
    assert np.allclose(orc.fft2(x), orc.dft2_naive(x), rtol=0, atol=1e-12 * np.abs(x).sum())
    assert np.allclose(orc.ifft2(orc.fft2(x)), x, atol=1e-13)


def test_parseval_and_sign_convention():
    g = synth.rng(2)
    x = _rand_c(g, (16, 16))
    assert np.isclose(np.linalg.norm(orc.fft2(x)), np.linalg.norm(x), rtol=1e-13)
    # forward kernel exp(-2 pi i k n / M): a plane wave exp(+2 pi i n/M) lands on k = 1
    n = np.arange(16)
    wave = np.exp(2j * np.pi * n / 16)[None, :] * np.ones((16, 1))
    F = orc.fft2(wave)
    assert np.isclose(abs(F[0, 1]), 16.0) and np.abs(F).sum() - 16.0 < 1e-9


def test_propagator_unitary_and_composes():
    g = synth.rng(3)
    x = _rand_c(g, (32, 32))
    h1 = orc.fresnel_propagator(32, 0.0251, 1.5, 0.1)
    h2 = orc.fresnel_propagator(32, 0.0251, 2.5, 0.1)
    h12 = orc.fresnel_propagator(32, 0.0251, 4.0, 0.1)
    assert np.allclose(np.abs(h1), 1.0)
    assert np.isclose(np.linalg.norm(orc.propagate(x, h1)), np.linalg.norm(x), rtol=1e-13)
    assert np.allclose(orc.propagate(orc.propagate(x, h1), h2), orc.propagate(x, h12), atol=1e-12)


def test_propagator_matches_gaussian_beam_closed_form():
    """Continuous Fresnel propagation of a Gaussian: u_z = (2 pi s^2)(pi/a) exp(-pi^2 r^2 / a),
    a = 2 pi^2 s^2 + i pi lambda z  (transfer function exp(-i pi lambda z |k|^2))."""
    M, px, s, lam, z = 128, 0.1, 0.6, 0.0251, 40.0
    c = np.arange(M) - M // 2
    y, x = np.meshgrid(c * px, c * px, indexing="ij")
    r2 = x * x + y * y
    u0 = np.exp(-r2 / (2 * s * s))
    # shift to FFT origin, propagate, shift back
    h = orc.fresnel_propagator(M, lam, z, px)
    uz = np.fft.fftshift(orc.propagate(np.fft.ifftshift(u0), h))
    a = 2 * np.pi ** 2 * s * s + 1j * np.pi * lam * z
    expect = (2 * np.pi * s * s) * (np.pi / a) * np.exp(-np.pi ** 2 * r2 / a)
    assert np.max(np.abs(uz - expect)) < 1e-9


def test_adjoints_by_dot_product():
    g = synth.rng(4)
    x, y = _rand_c(g, (12, 12)), _rand_c(g, (12, 12))
    h = orc.fresnel_propagator(12, 0.0251, 2.0, 0.1)
    ip = lambda a, b: np.vdot(a, b)
    assert np.isclose(ip(orc.fft2(x), y), ip(x, orc.ifft2(y)), rtol=1e-12)
    prop_adj = lambda v: orc.ifft2(np.conj(h) * orc.fft2(v))
    assert np.isclose(ip(orc.propagate(x, h), y), ip(x, prop_adj(y)), rtol=1e-12)


# ---------------------------------------------------------------- loss (Eq. 1)

def test_zero_loss_and_gradient_at_truth():
    probe, obj, pos, _, h = _small_problem(noise=False)
    I = orc.intensities(probe, obj, pos, h)
    L, gO, gP = orc.loss_grad(probe, obj, pos, I, h)
    assert L < 1e-20 * I.sum()
    assert np.abs(gO).max() < 1e-9 and np.abs(gP).max() < 1e-9


def test_vacuum_reduces_to_single_fft():
    """O_s = 1: the propagators only multiply the spectrum by |h| = 1 phases,
    so |Psi| = |F P| independent of S and dz; the loss is the textbook sum."""
    g = synth.rng(5)
    M, S, H, W = 8, 4, 12, 12
    probe = _rand_c(g, (M, M))
    obj = np.ones((S, H, W), complex)
    pos = np.array([[0, 0], [2, 3], [4, 4]], np.int32)
    I = g.uniform(0, 5, (3, M, M))
    h = orc.fresnel_propagator(M, 0.0251, 7.0, 0.1)
    expect = sum(np.sum((np.abs(np.fft.fft2(probe) / M) - np.sqrt(I[i])) ** 2) for i in range(3))
    assert np.isclose(orc.loss(probe, obj, pos, I, h), expect, rtol=1e-12)


def test_extra_propagation_after_last_slice_changes_nothing():
    probe, obj, pos, I, h = _small_problem()
    L = orc.loss(probe, obj, pos, I, h)
    L2 = 0.0
    for i, r in enumerate(pos):
        _, phi, _ = orc.multislice_waves(probe, obj, r, h)
        L2 += np.sum((np.abs(orc.fft2(orc.propagate(phi[-1], h))) - np.sqrt(I[i])) ** 2)
    assert np.isclose(L, L2, rtol=1e-12)


def test_invariances():
    probe, obj, pos, I, h = _small_problem()
    L = orc.loss(probe, obj, pos, I, h)
    ph = np.exp(0.7j)
    obj2 = obj.copy(); obj2[1] *= ph
    assert np.isclose(orc.loss(probe, obj2, pos, I, h), L, rtol=1e-12)
    assert np.isclose(orc.loss(probe * ph, obj, pos, I, h), L, rtol=1e-12)
    obj3 = obj.copy(); obj3[2] /= 1.7
    assert np.isclose(orc.loss(probe * 1.7, obj3, pos, I, h), L, rtol=1e-12)
    # shifting object and all positions together
    objs = np.zeros((obj.shape[0], obj.shape[1] + 3, obj.shape[2] + 2), complex)
    objs[:, 3:, 2:] = obj
    assert np.isclose(orc.loss(probe, objs, pos + np.array([3, 2], np.int32), I, h), L, rtol=1e-12)


# ---------------------------------------------------------------- gradient (Eq. 2)

def test_central_finite_differences():
    probe, obj, pos, I, h = _small_problem()
    L, gO, gP = orc.loss_grad(probe, obj, pos, I, h)
    g = synth.rng(11)
    eps = 1e-6
    for _ in range(8):
        dO = _rand_c(g, obj.shape)
        dP = _rand_c(g, probe.shape)
        fd = (orc.loss(probe + eps * dP, obj + eps * dO, pos, I, h)
              - orc.loss(probe - eps * dP, obj - eps * dO, pos, I, h)) / (2 * eps)
        an = np.real(np.vdot(gO, dO) + np.vdot(gP, dP))
        assert abs(fd - an) <= RTOL_FD * max(abs(an), 1e-3 * L), (fd, an)


def test_single_slice_gradient_by_explicit_jacobian():
    """S = 1: Psi_i = D diag(P) E_i o with D the 2-D DFT matrix (Kronecker of
    1-D DFT matrices) and E_i the window selection; g_o = sum E_i^T diag(conj P) D^H g_Psi,
    g_P = sum diag(conj(E_i o)) D^H g_Psi.  Built from dense matrices here."""
    g = synth.rng(12)
    M, H, W = 6, 9, 10
    probe = _rand_c(g, (M, M))
    obj = (1 + 0.2 * g.uniform(-1, 1, (1, H, W))) * np.exp(1j * g.uniform(-1, 1, (1, H, W)))
    pos = np.array([[0, 0], [3, 1], [2, 4], [1, 3]], np.int32)
    I = g.uniform(0.1, 4.0, (len(pos), M, M))
    h = orc.fresnel_propagator(M, 0.0251, 2.0, 0.1)
    n = np.arange(M)
    F1 = np.exp(-2j * np.pi * np.outer(n, n) / M) / np.sqrt(M)
    D = np.kron(F1, F1)
    o = obj[0].ravel()
    go = np.zeros(H * W, complex)
    gp = np.zeros(M * M, complex)
    Ltot = 0.0
    for i, (y, x) in enumerate(pos):
        E = np.zeros((M * M, H * W))
        for a in range(M):
            for b in range(M):
                E[a * M + b, (y + a) * W + (x + b)] = 1.0
        u = E @ o
        Psi = D @ (probe.ravel() * u)
        amp = np.abs(Psi)
        res = amp - np.sqrt(I[i].ravel())
        Ltot += np.sum(res ** 2)
        gPsi = 2 * res * Psi / amp
        back = D.conj().T @ gPsi
        go += E.T @ (np.conj(probe.ravel()) * back)
        gp += np.conj(u) * back
    L, gO, gP = orc.loss_grad(probe, obj, pos, I, h)
    assert np.isclose(L, Ltot, rtol=1e-12)
    assert np.allclose(gO[0].ravel(), go, atol=1e-10)
    assert np.allclose(gP.ravel(), gp, atol=1e-10)


def _multislice_problem(S, seed):
    """Tiny window, strong propagation (phases up to ~4 rad at the band edge),
    non-unimodular slices that differ from one another."""
    g = synth.rng(seed)
    M, H, W = 6, 10, 11
    probe = _rand_c(g, (M, M))
    obj = (1 + 0.3 * g.uniform(-1, 1, (S, H, W))) * np.exp(1j * g.uniform(-1.2, 1.2, (S, H, W)))
    pos = np.array([[0, 0], [4, 1], [2, 5], [3, 3]], np.int32)
    I = g.uniform(0.1, 4.0, (len(pos), M, M))
    geo = (0.0251, 2.0, 0.1)
    return probe, obj, pos, I, orc.fresnel_propagator(M, *geo), dm.fresnel_diag(M, *geo)


def check_against_dense(probe, obj, pos, I, h, hd):
    """The oracle's far fields, loss and gradients against the dense-matrix
    product of Sec. II-B's multislice model (tests/dense_multislice.py)."""
    far = orc.forward(probe, obj, pos, h)
    for i, r in enumerate(pos):
        _, Psi, _, _ = dm.position(probe, obj, r, I[i], hd)
        assert np.allclose(far[i].ravel(), Psi, rtol=0, atol=1e-12 * np.abs(Psi).max())
    L, gO, gP = orc.loss_grad(probe, obj, pos, I, h)
    Ld, gOd, gPd = dm.loss_grad(probe, obj, pos, I, hd)
    assert np.isclose(L, Ld, rtol=1e-12)
    assert np.allclose(gO, gOd, rtol=0, atol=1e-11 * np.abs(gOd).max())
    assert np.allclose(gP, gPd, rtol=0, atol=1e-11 * np.abs(gPd).max())


@pytest.mark.parametrize("S", [2, 3])
def test_multislice_composition_by_dense_matrices(S):
    """S >= 2 (Sec. II-B: the output of one slice is the input of the next):
    Psi = D T_{S-1} D^H diag(h) D ... T_1 D^H diag(h) D T_0 P with explicit
    matrices fixes the slice order, that each transmission precedes the
    propagation, and the adjoint of the whole chain (g = J^H g_Psi)."""
    check_against_dense(*_multislice_problem(S, 40 + S))


ARMIJO_CASES = [(1.0, 1e-3, "halved"), (1e-5, 1e-6, "full")]


def check_armijo(step_fn, aO, aP, expect):
    """Brute force over t = 1, 1/2, 1/4, ...: step_fn must return the first t
    with F(x - t a g) <= F(x) - 1e-4 t (a_O |g_O|^2 + a_P |g_P|^2).  The long
    steps need several halvings (a slip that accepts the first halving, or
    halves once too often, fails); with the short steps t = 1 passes while the
    same test with the step sizes left out of the decrease term accepts no t."""
    probe, obj, pos, I, h = _small_problem()
    L0, gO, gP = orc.loss_grad(probe, obj, pos, I, h)
    nO, nP = np.sum(np.abs(gO) ** 2), np.sum(np.abs(gP) ** 2)
    ts = [0.5 ** k for k in range(21)]
    F = {t: orc.loss(probe - t * aP * gP, obj - t * aO * gO, pos, I, h) for t in ts}
    first = next(t for t in ts if F[t] <= L0 - 1e-4 * t * (aO * nO + aP * nP))
    if expect == "halved":
        assert first <= 0.125
    else:
        assert first == 1.0
        assert not any(F[t] <= L0 - 1e-4 * t * (nO + nP) for t in ts)
    Pn, On, F0, t = step_fn(probe, obj, pos, I, h, aO, aP, line_search=True)
    assert F0 == L0 and t == first
    assert np.allclose(On, obj - t * aO * gO, rtol=0, atol=1e-14)
    assert np.allclose(Pn, probe - t * aP * gP, rtol=0, atol=1e-14)


@pytest.mark.parametrize("aO, aP, expect", ARMIJO_CASES)
def test_armijo_accepts_the_first_passing_halving(aO, aP, expect):
    check_armijo(orc.step, aO, aP, expect)


def test_orthogonality_identities():
    """Global phase and probe/object scale exchange leave Eq. 1 invariant, so
    Re<g_O_s, i O_s> = 0, Re<g_P, i P> = 0 and Re<g_P, P> = Re<g_O_s, O_s> per slice."""
    probe, obj, pos, I, h = _small_problem()
    _, gO, gP = orc.loss_grad(probe, obj, pos, I, h)
    scale = np.abs(gP).sum() * np.abs(probe).sum()
    assert abs(np.real(np.vdot(gP, 1j * probe))) < 1e-10 * scale
    for s in range(obj.shape[0]):
        assert abs(np.real(np.vdot(gO[s], 1j * obj[s]))) < 1e-10 * scale
        assert np.isclose(np.real(np.vdot(gP, probe)), np.real(np.vdot(gO[s], obj[s])),
                          rtol=1e-10, atol=1e-10 * scale)


def test_locality_and_batch_invariance():
    """Sec. III: each position's gradient is supported on its window; Eq. 2: the
    gradient over any partition of the positions sums to the full gradient."""
    probe, obj, pos, I, h = _small_problem(N=6)
    L, gO, gP = orc.loss_grad(probe, obj, pos, I, h)
    M = probe.shape[0]
    for i in range(len(pos)):
        Li, gOi, _ = orc.loss_grad(probe, obj, pos[i:i + 1], I[i:i + 1], h)
        mask = np.zeros(obj.shape[1:], bool)
        y, x = pos[i]
        mask[y:y + M, x:x + M] = True
        assert np.all(gOi[:, ~mask] == 0)
    parts = [[0, 3], [1, 4, 5], [2]]
    acc = [0.0, np.zeros_like(gO), np.zeros_like(gP)]
    for p in parts:
        Lp, gOp, gPp = orc.loss_grad(probe, obj, pos[p], I[p], h)
        acc[0] += Lp; acc[1] += gOp; acc[2] += gPp
    assert np.isclose(acc[0], L, rtol=1e-13)
    assert np.allclose(acc[1], gO, atol=1e-12) and np.allclose(acc[2], gP, atol=1e-12)


def test_zero_amplitude_subgradient():
    Psi = np.array([[0.0 + 0j, 1 + 1j]])
    I = np.array([[4.0, 2.0]])
    g = orc.amplitude_residual_grad(Psi, I)
    assert g[0, 0] == 0 and np.isclose(g[0, 1], 0.0)


def test_potential_gradient_finite_difference():
    probe, obj, pos, I, h = _small_problem()
    V = np.real(-1j * np.log(obj / np.abs(obj)))
    amp = np.abs(obj)
    sigma = 0.8
    V = V / sigma
    mk = lambda VV: amp * np.exp(1j * sigma * VV)
    _, gO, _ = orc.loss_grad(probe, mk(V), pos, I, h)
    gV = orc.potential_grad(mk(V), gO, sigma)
    g = synth.rng(13)
    d = g.standard_normal(V.shape)
    eps = 1e-6
    fd = (orc.loss(probe, mk(V + eps * d), pos, I, h) - orc.loss(probe, mk(V - eps * d), pos, I, h)) / (2 * eps)
    assert np.isclose(fd, np.sum(gV * d), rtol=1e-7)


def test_step_fixed_and_armijo():
    probe, obj, pos, I, h = _small_problem()
    L0, gO, gP = orc.loss_grad(probe, obj, pos, I, h)
    Pn, On, F0, t = orc.step(probe, obj, pos, I, h, 1e-3, 1e-4)
    assert F0 == L0 and t == 1.0
    assert np.allclose(On, obj - 1e-3 * gO) and np.allclose(Pn, probe - 1e-4 * gP)
    Pn, On, F0, t = orc.step(probe, obj, pos, I, h, 10.0, 10.0, line_search=True)
    assert 0 < t < 1
    assert orc.loss(Pn, On, pos, I, h) < L0


def test_out_of_bounds_positions_rejected():
    probe, obj, pos, I, h = _small_problem()
    bad = pos.copy(); bad[0, 1] = obj.shape[2] - probe.shape[0] + 1
    with pytest.raises(ValueError):
        orc.loss_grad(probe, obj, bad, I, h)
