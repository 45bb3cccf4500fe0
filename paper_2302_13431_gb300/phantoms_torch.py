"""The synthetic calibration recipe of phantoms.make_case evaluated on the GPU with torch, for
generating many training volumes quickly (the warm start's training set).

Every random parameter (ellipsoid centres, axes, rotations, amplitudes, coil phase
coefficients) is drawn from numpy's default_rng(seed) in the same order as make_case; the
arrays are built in FP64 on the device; only the k-space noise comes from a seeded torch
generator, so the noise differs from make_case's (the parity tests keep using make_case).
This module holds input generation only: none of the estimator's arithmetic.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from .phantoms import _ring_centres


def _axes(shape, device):
    return [(torch.arange(n, device=device, dtype=torch.float64) - n // 2) / n for n in shape]


def _mesh(shape, device):
    return torch.meshgrid(*_axes(shape, device), indexing="ij")


def make_calib(grid, Q, calib_shape, seed=0, noise=0.01, phase="poly4", sigma=0.35, radius=0.6,
               n_ellipses=10, device="cuda"):
    """complex64 calibration block [Q][Nc...] (and the phantom) on `device`."""
    rng = np.random.default_rng(seed)
    grid = tuple(int(g) for g in grid)
    D = len(grid)
    X = _mesh(grid, device)
    xs = X[::-1]  # x, y, (z)
    pts = torch.stack([a.reshape(-1) for a in xs], dim=1)
    img = torch.zeros(pts.shape[0], dtype=torch.complex128, device=device)
    for _ in range(n_ellipses):
        c = rng.uniform(-0.15, 0.15, D)
        ax = rng.uniform(0.05, 0.25, D)
        M = rng.standard_normal((D, D))
        Qm, Rm = np.linalg.qr(M)
        Qm = Qm * np.sign(np.diag(Rm))
        amp = rng.uniform(0.2, 1.0) * np.exp(1j * rng.uniform(0.0, 2 * np.pi))
        local = (pts - torch.from_numpy(c).to(device)) @ torch.from_numpy(Qm).to(device)
        inside = torch.sum((local / torch.from_numpy(ax).to(device)) ** 2, dim=1) <= 1.0
        img[inside] += complex(amp)
    rho = img.reshape(grid)
    cen = _ring_centres(Q, D, radius)
    degree = 1 if phase == "linear" else 4
    exps = [e for e in np.ndindex(*([degree + 1] * D)) if sum(e) <= degree]
    maps = torch.empty((Q,) + grid, dtype=torch.complex128, device=device)
    for q in range(Q):
        r2 = sum((xs[d] - float(cen[q, d])) ** 2 for d in range(D))
        mag = torch.exp(-r2 / (2 * sigma ** 2))
        ph = torch.zeros(grid, dtype=torch.float64, device=device)
        for e in exps:
            coef = rng.normal(0.0, 2.0 / math.factorial(sum(e)))
            term = torch.ones(grid, dtype=torch.float64, device=device)
            for d in range(D):
                if e[d]:
                    term = term * xs[d] ** e[d]
            ph = ph + coef * term
        maps[q] = mag * torch.exp(1j * ph)
    maps = maps / torch.sqrt(torch.sum(maps.abs() ** 2, dim=0))
    axes = tuple(range(1, D + 1))
    k = torch.fft.fftshift(torch.fft.fftn(torch.fft.ifftshift(maps * rho[None], dim=axes), dim=axes), dim=axes)
    del maps
    sl = [slice(None)]
    for n, nc in zip(grid, calib_shape):
        s = n // 2 - nc // 2
        sl.append(slice(s, s + nc))
    kc = k[tuple(sl)].clone()
    if noise > 0:
        sig = noise * float(k.abs().max())
        g = torch.Generator(device=device)
        g.manual_seed(int(seed) + 0x5EED)
        kc = kc + (sig / math.sqrt(2.0)) * torch.complex(
            torch.randn(kc.shape, generator=g, device=device, dtype=torch.float64),
            torch.randn(kc.shape, generator=g, device=device, dtype=torch.float64))
    del k
    return kc.to(torch.complex64).contiguous(), rho
