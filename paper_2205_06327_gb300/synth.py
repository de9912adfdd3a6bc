"""Seeded synthetic inputs shaped like the paper's workloads.

The paper evaluates on simulated PbTiO3 datasets (Sec. VI-A, Table I) that are
not distributed with it.  This module builds stand-ins with the same
structure: a raster scan of probe positions with heavy overlap (Fig. 3), a
defocused probe from a circular aperture, and a stack of complex
transmission slices O_s = exp(i*sigma*V_s) of a Gaussian-atom potential.

Nothing here evaluates the multislice model, the loss or its gradient: the
measured intensities are made by whoever consumes these inputs (the oracle in
the tests, ``ptycho_forward`` in the benchmark); the only randomness of the
measurement, the Poisson counts, is drawn here from a seeded generator.

All arrays are numpy complex128 / float64 / int32; callers cast as needed.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# Seeds: workload j of the five shapes below uses 1000 + j; problem p of the
# batched workload uses 5000 + p.
SEED_BASE = 1000
MULTI_SEED_BASE = 5000


@dataclass
class Workload:
    """One reconstruction problem: everything except the measured intensities."""

    name: str
    M: int                      # probe window (square), detector pixels per side
    S: int                      # number of slices
    H: int                      # object height (pixels)
    W: int                      # object width (pixels)
    pos: np.ndarray             # int32 [N, 2] top-left (y, x) of each window, raster order
    probe: np.ndarray           # complex128 [M, M]
    obj: np.ndarray             # complex128 [S, H, W] transmissions
    lambda_A: float = 0.0251    # electron wavelength (Angstrom)
    dz_A: float = 2.0           # slice spacing (Angstrom)
    pixel_A: float = 0.1        # real-space pixel (Angstrom)
    sigma: float = 1.0          # interaction constant; V is pre-scaled so sigma = 1
    counts: float | None = None  # Poisson dose per pattern (None = noise-free)
    potential: np.ndarray | None = None  # float64 [S, H, W] V (O = exp(i sigma V))
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.pos.shape[0])


def rng(seed: int) -> np.random.Generator:
    """The one generator every seeded input uses (PCG64)."""
    return np.random.Generator(np.random.PCG64(seed))


def raster_positions(ny: int, nx: int, step: int, y0: int, x0: int) -> np.ndarray:
    """Raster scan, x fastest (Fig. 3 caption), integer top-left corners."""
    ys = y0 + step * np.arange(ny)
    xs = x0 + step * np.arange(nx)
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    return np.stack([yy.ravel(), xx.ravel()], axis=1).astype(np.int32)


def _freq_grid(M: int, d: float):
    k = np.fft.fftfreq(M, d=d)
    return k[:, None], k[None, :]


def defocused_probe(M: int, k_aperture: float, chi_coeff: float, d: float,
                    energy: float = 1.0) -> np.ndarray:
    """Probe = inverse FFT of A(k) exp(-i chi(k)), chi = chi_coeff*|k|^2.

    A is a hard circular aperture |k| <= k_aperture; k = fftfreq(M, d).  The
    probe is centred in the window and scaled to total energy ``energy``.
    """
    ky, kx = _freq_grid(M, d)
    k2 = ky * ky + kx * kx
    A = (k2 <= k_aperture * k_aperture).astype(np.float64)
    spec = A * np.exp(-1j * chi_coeff * k2)
    p = np.fft.ifft2(spec)
    p = np.fft.fftshift(p)
    p *= np.sqrt(energy / np.sum(np.abs(p) ** 2))
    return p


def _splat_gaussians(H: int, W: int, centers: np.ndarray, weights: np.ndarray,
                     sigma_px: float) -> np.ndarray:
    """Sum of isotropic Gaussians (unit peak times weight), rendered locally."""
    img = np.zeros((H, W))
    r = int(np.ceil(5 * sigma_px))
    off = np.arange(-r, r + 1)
    for (cy, cx), w in zip(centers, weights):
        iy, ix = int(np.floor(cy)), int(np.floor(cx))
        ys = iy + off
        xs = ix + off
        my = (ys >= 0) & (ys < H)
        mx = (xs >= 0) & (xs < W)
        if not my.any() or not mx.any():
            continue
        gy = np.exp(-0.5 * ((ys[my] - cy) / sigma_px) ** 2)
        gx = np.exp(-0.5 * ((xs[mx] - cx) / sigma_px) ** 2)
        img[np.ix_(ys[my], xs[mx])] += w * gy[:, None] * gx[None, :]
    return img


def _scale_to_max(V: np.ndarray, max_phase: float) -> np.ndarray:
    """Scale each slice so that its maximum is ``max_phase`` (sigma = 1)."""
    out = np.empty_like(V)
    for s in range(V.shape[0]):
        m = V[s].max()
        out[s] = V[s] * (max_phase / m) if m > 0 else V[s]
    return out


def workload_single_slice(seed: int = SEED_BASE + 1) -> Workload:
    """Single-slice 2-D case: 192^2 phase object, 64^2 probe, 8x8 raster, step 12."""
    g = rng(seed)
    H = W = 192
    lat = np.arange(3, H, 6, dtype=np.float64)
    cy, cx = np.meshgrid(lat, lat, indexing="ij")
    centers = np.stack([cy.ravel(), cx.ravel()], 1)
    centers = centers + g.uniform(-1.0, 1.0, size=centers.shape)
    V = _splat_gaussians(H, W, centers, np.ones(len(centers)), 1.5)[None]
    V = _scale_to_max(V, 0.5)
    M = 64
    # geometric defocus disc of 50 px: 2 * lambda*df * k_ap = 50 with
    # k_ap = 12/64 cycles/px  ->  lambda*df = 133.33 px^2
    k_ap = 12.0 / M
    ldf = 50.0 / (2.0 * k_ap)
    probe = defocused_probe(M, k_ap, np.pi * ldf, 1.0, energy=1.0)
    pos = raster_positions(8, 8, 12, 22, 22)
    return Workload("single-slice 64^2 window, 192^2 object, 64 positions",
                    M, 1, H, W, pos, probe, np.exp(1j * V), dz_A=2.0,
                    potential=V, counts=None)


def workload_multislice(seed: int = SEED_BASE + 2) -> Workload:
    """16 slices of 384^2, 128^2 probe (20 mrad, 100 A defocus), 24x24 raster step 10."""
    g = rng(seed)
    S, H, W, M = 16, 384, 384, 128
    lam, px = 0.0251, 0.1
    lat = np.arange(10, H, 20, dtype=np.float64)
    cy, cx = np.meshgrid(lat, lat, indexing="ij")
    sites = np.stack([cy.ravel(), cx.ravel()], 1)
    V = np.empty((S, H, W))
    for s in range(S):
        occ = g.random(len(sites)) < 0.5
        V[s] = _splat_gaussians(H, W, sites[occ], np.ones(int(occ.sum())), 3.0)
    V = _scale_to_max(V, 0.3)
    k_ap = 0.020 / lam
    probe = defocused_probe(M, k_ap, np.pi * lam * 100.0, px, energy=1.0e4)
    pos = raster_positions(24, 24, 10, 13, 13)
    return Workload("multislice 128^2 window, 16 x 384^2 object, 576 positions",
                    M, S, H, W, pos, probe, np.exp(1j * V), lambda_A=lam, dz_A=2.0,
                    pixel_A=px, potential=V, counts=1.0e4)


def workload_perovskite(seed: int = SEED_BASE + 3, n_rows: int = 126,
                        n_cols: int = 132) -> Workload:
    """PbTiO3-shaped: 30 x 640x656 object, 128^2 probe, 126x132 raster step 4."""
    g = rng(seed)
    S, H, W, M = 30, 640, 656, 128
    lam, px, a = 0.0251, 0.1, 39.0
    cells_y = np.arange(-1, int(H / a) + 2)
    cells_x = np.arange(-1, int(W / a) + 2)
    shift = g.uniform(0.0, a, size=2)
    cyy, cxx = np.meshgrid(cells_y * a + shift[0], cells_x * a + shift[1], indexing="ij")
    corner = np.stack([cyy.ravel(), cxx.ravel()], 1)
    centre = corner + a / 2
    edge_y = corner + np.array([a / 2, 0.0])
    edge_x = corner + np.array([0.0, a / 2])
    V = np.empty((S, H, W))
    for s in range(S):
        if s % 2 == 0:     # PbO layer: Pb at corners, O at the face centre
            c = np.concatenate([corner, centre])
            w = np.concatenate([np.full(len(corner), 82.0), np.full(len(centre), 8.0)])
        else:              # TiO2 layer: Ti at the centre, O at the edge centres
            c = np.concatenate([centre, edge_y, edge_x])
            w = np.concatenate([np.full(len(centre), 22.0), np.full(2 * len(edge_y), 8.0)])
        V[s] = _splat_gaussians(H, W, c, w, 3.0)
    V = _scale_to_max(V, 0.3)
    k_ap = 0.030 / lam
    probe = defocused_probe(M, k_ap, np.pi * lam * 250.0, px, energy=1.0e5)
    pos = raster_positions(n_rows, n_cols, 4, 6, 2)
    return Workload("PbTiO3-shaped 128^2 window, 30 x 640x656 object, "
                    f"{n_rows * n_cols} positions",
                    M, S, H, W, pos, probe, np.exp(1j * V), lambda_A=lam, dz_A=1.25,
                    pixel_A=px, potential=V, counts=1.0e5)


def workload_paper_scale(S: int = 100, n_pos: int = 8, seed: int = SEED_BASE + 6) -> Workload:
    """The paper's per-position shape (Table I: 1024^2 detector, 100 slices) on
    a short diagonal scan: positions 8 px apart in y and 16 px in x, a smooth
    random phase object (band-limited Gaussian noise scaled to 0.3 rad per
    slice; generated with FFTs, unlike the atom splatting above, which would
    take minutes at this size), the defocused probe of :func:`workload_random`.
    Noise-free data (the caller scales or perturbs them)."""
    M = 1024
    g = rng(seed)
    H, W = M + 8 * (n_pos - 1) + 2, M + 16 * (n_pos - 1) + 3
    ky = np.fft.fftfreq(H)[:, None]
    kx = np.fft.fftfreq(W)[None, :]
    lowpass = np.exp(-(ky ** 2 + kx ** 2) / (2 * 0.02 ** 2))
    obj = np.empty((S, H, W), np.complex64)
    for s in range(S):
        ph = np.fft.ifft2(np.fft.fft2(g.standard_normal((H, W))) * lowpass).real
        obj[s] = np.exp(1j * 0.3 * ph / np.abs(ph).max())
    probe = defocused_probe(M, 0.15, np.pi * 0.15 * M, 1.0, energy=float(M))
    pos = np.array([[8 * i, 16 * i] for i in range(n_pos)], np.int32)
    return Workload(f"paper-scale 1024^2 window, {S} x {H}x{W} object, {n_pos} positions", M, S, H, W, pos,
                    probe, obj)


def workload_random(M: int, S: int, ny: int, nx: int, step: int, seed: int,
                    max_phase: float = 0.3, amp_jitter: float = 0.0,
                    counts: float | None = None) -> Workload:
    """Small generic problem (tests): random smooth phase slices, defocused probe.

    ``amp_jitter`` > 0 makes the transmissions non-unimodular
    (|O| = 1 + amp_jitter*u, u uniform in [-1, 1]), which exercises the
    adjoint of the transmission for general complex O.
    """
    g = rng(seed)
    H = (ny - 1) * step + M + 2
    W = (nx - 1) * step + M + 3
    n_atoms = max(4, (H * W) // 36)
    V = np.empty((S, H, W))
    for s in range(S):
        c = np.stack([g.uniform(0, H, n_atoms), g.uniform(0, W, n_atoms)], 1)
        V[s] = _splat_gaussians(H, W, c, g.uniform(0.5, 1.0, n_atoms), 1.5)
    V = _scale_to_max(V, max_phase)
    O = np.exp(1j * V)
    if amp_jitter > 0:
        O = O * (1.0 + amp_jitter * g.uniform(-1.0, 1.0, size=O.shape))
    k_ap = 0.3 * 0.5  # cycles/px
    probe = defocused_probe(M, k_ap, np.pi * 0.15 * M, 1.0, energy=float(M))
    pos = raster_positions(ny, nx, step, 1, 2)
    lam, px = 0.0251, 0.1
    return Workload(f"random M={M} S={S} N={ny * nx}", M, S, H, W, pos, probe, O,
                    lambda_A=lam, dz_A=2.0, pixel_A=px, potential=V, counts=counts)


def workload(config_id: int) -> Workload:
    """The workload shapes by number (1: single slice, 2/4: multislice,
    3: PbTiO3-shaped, 6: the paper's per-position shape on 8 positions)."""
    if config_id == 1:
        return workload_single_slice()
    if config_id in (2, 4):
        return workload_multislice()
    if config_id == 3:
        return workload_perovskite()
    if config_id == 6:
        return workload_paper_scale()
    raise ValueError(f"no workload {config_id}")


def multi_problem_shapes(n_problems: int = 32, seed: int = MULTI_SEED_BASE):
    """Shapes of the batched uneven workload: (M, S, ny, nx, step) per problem.

    Windows from {64, 96, 128, 192, 256}, 256..4096 positions, 1..24 slices.
    """
    g = rng(seed)
    shapes = []
    for p in range(n_problems):
        M = int(g.choice([64, 96, 128, 192, 256]))
        S = int(g.integers(1, 25))
        n = int(g.integers(256, 4097))
        ny = int(np.floor(np.sqrt(n)))
        nx = int(np.ceil(n / ny))
        step = max(2, M // 16)
        shapes.append((M, S, ny, nx, step))
    return shapes


def poisson_counts(intensity: np.ndarray, seed: int) -> np.ndarray:
    """Poisson-distributed counts with mean ``intensity`` (float32 result)."""
    g = rng(seed + 100)
    return g.poisson(np.maximum(intensity, 0.0)).astype(np.float32)
