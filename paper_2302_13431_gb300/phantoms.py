"""Seeded synthetic multichannel calibration data.

This module only generates inputs: an ellipse/ellipsoid phantom rho(x), smooth coil
sensitivities c_q(x), and Nyquist-sampled multichannel k-space following the forward
model of Eq. (1) (d_q(k) = FT{c_q rho}(k) + noise), discretised on the image grid with
the FOV normalised to the unit cube (Sec. III-A).  It holds none of the estimator's
arithmetic, so both the CUDA path and the CPU oracle can consume what it produces.

Grid convention (shared by every consumer): an axis of length N holds the points
x_j = (j - N//2) / N, j = 0..N-1, and the k-space index n_j = j - N//2 (DC at N//2).
Arrays are C-ordered with x fastest: images are [Nz][Ny][Nx] (Nz absent in 2D) and
multichannel arrays put the coil index first.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "grid_coords", "ellipse_phantom", "coil_maps", "centered_dft", "add_noise",
    "crop_center", "SyntheticCase", "make_case", "PAPER_WORKLOADS", "uneven_slice_specs",
]


def grid_coords(shape):
    """Per-axis coordinates x_j = (j - N//2)/N for an image of `shape` (z,y,x order)."""
    return [(np.arange(n) - n // 2) / n for n in shape]


def _mesh(shape):
    return np.meshgrid(*grid_coords(shape), indexing="ij")


def ellipse_phantom(shape, rng, n_ellipses=10):
    """Sum of `n_ellipses` random ellipses (2D) or ellipsoids (3D).

    Centres U[-0.15,0.15]^D, semi-axes U[0.05,0.25], random orientation, intensities
    U[0.2,1] and phases U[0,2pi).  Every shape lies inside |x|_inf < 0.4, so the support
    Omega is strictly inside the FOV, as the limited-support argument of Sec. III-A needs.
    """
    D = len(shape)
    X = _mesh(shape)
    pts = np.stack([a.reshape(-1) for a in X[::-1]], axis=1)  # (npix, D) in x,y,z order
    img = np.zeros(pts.shape[0], dtype=np.complex128)
    for _ in range(n_ellipses):
        c = rng.uniform(-0.15, 0.15, D)
        ax = rng.uniform(0.05, 0.25, D)
        # random rotation: QR of a Gaussian matrix with a sign fix
        M = rng.standard_normal((D, D))
        Qm, Rm = np.linalg.qr(M)
        Qm = Qm * np.sign(np.diag(Rm))
        amp = rng.uniform(0.2, 1.0) * np.exp(1j * rng.uniform(0.0, 2 * np.pi))
        local = (pts - c) @ Qm
        inside = np.sum((local / ax) ** 2, axis=1) <= 1.0
        img[inside] += amp
    return img.reshape(shape)


def _ring_centres(Q, D, radius):
    if D == 2:
        ang = 2 * np.pi * np.arange(Q) / Q
        return np.stack([radius * np.cos(ang), radius * np.sin(ang)], axis=1)
    # Fibonacci sphere for 3D
    i = np.arange(Q) + 0.5
    phi = np.arccos(1 - 2 * i / Q)
    th = np.pi * (1 + 5 ** 0.5) * i
    return radius * np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], axis=1)


def coil_maps(shape, Q, rng, sigma=0.35, radius=0.6, phase="poly4"):
    """Q Gaussian-blob sensitivities centred on a ring (2D) or sphere (3D) of `radius`,
    width `sigma` (FOV units), times a smooth phase, normalised to unit root-sum-of-squares.

    phase="linear": a random linear phase; phase="poly4": a random polynomial phase of
    total degree 4 whose coefficient for a monomial of degree k is N(0, (2/k!)^2).
    """
    D = len(shape)
    X = _mesh(shape)
    xs = X[::-1]  # x, y, (z)
    cen = _ring_centres(Q, D, radius)
    maps = np.empty((Q,) + tuple(shape), dtype=np.complex128)
    degree = 1 if phase == "linear" else 4
    exps = [e for e in np.ndindex(*([degree + 1] * D)) if sum(e) <= degree]
    for q in range(Q):
        r2 = sum((xs[d] - cen[q, d]) ** 2 for d in range(D))
        mag = np.exp(-r2 / (2 * sigma ** 2))
        ph = np.zeros(shape)
        for e in exps:
            k = sum(e)
            coef = rng.normal(0.0, 2.0 / math.factorial(k))
            term = np.ones(shape)
            for d in range(D):
                term = term * xs[d] ** e[d]
            ph = ph + coef * term
        maps[q] = mag * np.exp(1j * ph)
    rss = np.sqrt(np.sum(np.abs(maps) ** 2, axis=0))
    return maps / rss


def centered_dft(img, axes):
    """Unnormalised DFT with the index origin at N//2 on every transformed axis:
    s[n] = sum_x f(x) exp(-i 2 pi n x), the discretisation of Eq. (1)."""
    return np.fft.fftshift(np.fft.fftn(np.fft.ifftshift(img, axes=axes), axes=axes), axes=axes)


def add_noise(k, rng, rel_sigma):
    """Complex Gaussian noise with E|eta|^2 = (rel_sigma * max|k|)^2 (each of the real and
    imaginary parts has standard deviation sigma/sqrt(2))."""
    sig = rel_sigma * np.max(np.abs(k))
    return k + (sig / np.sqrt(2.0)) * (rng.standard_normal(k.shape) + 1j * rng.standard_normal(k.shape))


def crop_center(k, calib_shape):
    """Central calibration box; its DC sits at index floor(Nc/2) on every axis."""
    sl = [slice(None)]
    for n, nc in zip(k.shape[1:], calib_shape):
        s = n // 2 - nc // 2
        sl.append(slice(s, s + nc))
    return k[tuple(sl)]


@dataclass
class SyntheticCase:
    calib: np.ndarray          # complex64 [Q][Nc...]
    rho: np.ndarray            # complex128 image
    maps: np.ndarray           # complex128 [Q][N...] true sensitivities
    grid: tuple
    calib_shape: tuple
    meta: dict = field(default_factory=dict)


def make_case(grid, Q, calib_shape, seed=0, noise=0.01, phase="poly4", sigma=0.35,
              n_ellipses=10):
    """One seeded case: phantom x maps -> centred DFT -> noise -> central crop."""
    rng = np.random.default_rng(seed)
    grid = tuple(int(g) for g in grid)
    rho = ellipse_phantom(grid, rng, n_ellipses)
    maps = coil_maps(grid, Q, rng, sigma=sigma, phase=phase)
    axes = tuple(range(1, len(grid) + 1))
    k = centered_dft(maps * rho[None], axes)
    if noise > 0:
        k = add_noise(k, rng, noise)
    calib = crop_center(k, calib_shape).astype(np.complex64)
    return SyntheticCase(calib=np.ascontiguousarray(calib), rho=rho, maps=maps, grid=grid,
                         calib_shape=tuple(calib_shape),
                         meta=dict(seed=seed, noise=noise, phase=phase, sigma=sigma))


# The paper's evaluation workloads restated as synthetic configurations (sizes only).
PAPER_WORKLOADS = {
    "2d_small": dict(grid=(64, 64), Q=8, calib=(24, 24), kernel="rect", tau=2, reduction=1,
                     iters=30, phase="linear"),
    "2d_256": dict(grid=(256, 256), Q=32, calib=(32, 32), kernel="ellipsoid", tau=3,
                   reduction=4, iters=30, phase="poly4"),
    "3d_128x128x96": dict(grid=(96, 128, 128), Q=32, calib=(24, 24, 24), kernel="ellipsoid",
                          tau=3, reduction=4, iters=30, phase="poly4"),
}


def uneven_slice_specs(count=96, seed=0):
    """Seeded shapes of the batched uneven-slice workload: square grids drawn uniformly from
    {192, 224, 256, 288, 320}, Q from {16, 32, 48, 64}, square calibration 24..40 (inclusive),
    ellipsoidal kernel of radius 3, grid reduction 4, 30 power iterations.  Each spec carries
    the seed of its own synthetic case (data seed = 5000 + index)."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        n = int(rng.choice([192, 224, 256, 288, 320]))
        q = int(rng.choice([16, 32, 48, 64]))
        c = int(rng.integers(24, 41))
        specs.append(dict(grid=(n, n), calib_shape=(c, c), num_coils=q, tau=3, kernel_shape="ellipsoid",
                          reduction=4, iters=30, data_seed=5000 + i))
    return specs

