"""The multislice model of Sec. II-B written out as a product of dense matrices.

Test infrastructure for the CPU pins.  For one position at corner r and tiny
windows (M <= 8) the far field is

    Psi = D diag(E_{S-1} o_{S-1}) D^H diag(h) D ... diag(E_1 o_1) D^H diag(h) D diag(E_0 o_0) P

with every factor a plain matrix: D the orthonormal 2-D DFT (the Kronecker
product of two 1-D DFT matrices, each entry exp(-2 pi i k n / M) / sqrt(M)),
diag(h) the Fresnel factor written from its definition, and E_s the 0/1
matrix that selects slice s's M x M window of the raveled object.  Slice 0
acts first on the probe, and each slice's transmission precedes the
propagation to the next (the output of one slice is the input of the next).

Nothing here calls the oracle or an FFT routine, so it pins the oracle's
composition of slices, not only each block on its own.
"""
from __future__ import annotations

import numpy as np


def dft_matrix(M: int) -> np.ndarray:
    """Orthonormal 2-D DFT of a raveled M x M array, (M^2, M^2)."""
    n = np.arange(M)
    f1 = np.exp(-2j * np.pi * np.outer(n, n) / M) / np.sqrt(M)
    return np.kron(f1, f1)


def fresnel_diag(M: int, lambda_A: float, dz_A: float, pixel_A: float) -> np.ndarray:
    """h(ky, kx) = exp(-i pi lambda dz (ky^2 + kx^2)) over raveled FFT-order
    frequencies: index j stands for j / (M pixel) up to (M - 1) / 2 and for
    (j - M) / (M pixel) above."""
    j = np.arange(M)
    f = np.where(j <= (M - 1) // 2, j, j - M) / (M * pixel_A)
    k2 = f[:, None] ** 2 + f[None, :] ** 2
    return np.exp(-1j * np.pi * lambda_A * dz_A * k2).ravel()


def window_matrix(r, M: int, H: int, W: int) -> np.ndarray:
    """E: (M^2, H W) 0/1 selection of the window with top-left corner r."""
    y, x = int(r[0]), int(r[1])
    E = np.zeros((M * M, H * W))
    for a in range(M):
        for b in range(M):
            E[a * M + b, (y + a) * W + (x + b)] = 1.0
    return E


def position(probe, obj, r, I_r, hdiag):
    """(f, Psi, J_obj, J_probe) for one position.

    J_obj[s] is the matrix of the linear map o_s -> Psi with the other
    unknowns held fixed, J_probe that of P -> Psi, so with
    g_Psi = 2 (|Psi| - sqrt(I)) Psi / |Psi| the gradients in the convention
    dL/dRe + i dL/dIm are J^H g_Psi.
    """
    S, H, W = obj.shape
    M = probe.shape[0]
    D = dft_matrix(M)
    Dh = D.conj().T
    Prop = Dh @ np.diag(hdiag) @ D            # free space between slices
    T = []                                     # transmissions, diag(E_s o_s)
    E = window_matrix(r, M, H, W)
    for s in range(S):
        T.append(np.diag(E @ obj[s].ravel()))
    # psi[s]: the wave entering slice s
    psi = [probe.ravel().astype(complex)]
    for s in range(S - 1):
        psi.append(Prop @ (T[s] @ psi[s]))
    Psi = D @ (T[S - 1] @ psi[S - 1])
    # after[s]: everything applied after slice s's transmission
    after = [None] * S
    after[S - 1] = D
    for s in range(S - 2, -1, -1):
        after[s] = after[s + 1] @ T[s + 1] @ Prop
    J_obj = [after[s] @ np.diag(psi[s]) @ E for s in range(S)]
    J_probe = after[0] @ T[0]
    amp = np.abs(Psi)
    res = amp - np.sqrt(I_r.ravel())
    return float(np.sum(res ** 2)), Psi, J_obj, J_probe


def loss_grad(probe, obj, pos, I, hdiag):
    """(F, dF/dO [S, H, W], dF/dP [M, M]) from the dense matrices."""
    S, H, W = obj.shape
    M = probe.shape[0]
    L = 0.0
    gO = np.zeros((S, H * W), complex)
    gP = np.zeros(M * M, complex)
    for i, r in enumerate(pos):
        f, Psi, J_obj, J_probe = position(probe, obj, r, I[i], hdiag)
        L += f
        amp = np.abs(Psi)
        gPsi = 2 * (amp - np.sqrt(I[i].ravel())) * Psi / amp
        for s in range(S):
            gO[s] += J_obj[s].conj().T @ gPsi
        gP += J_probe.conj().T @ gPsi
    return L, gO.reshape(S, H, W), gP.reshape(M, M)
