"""Whole-map runs of the FP64 oracle on all host cores, and the accuracy measure used against it.

TEST INFRASTRUCTURE ONLY, like the rest of `oracle/`: the test suite and the CPU-baseline /
reference legs of the benchmark use it; nothing in the product path imports it.

`estimate_parallel` computes exactly what `pisco_oracle.estimate` computes, with the same
functions in the same order: the calibration matrix and its FP64 SVD in this process, then the
per-pixel stages (G(x) = H(x)^H H(x) from explicit H(x), power iteration, phase) on disjoint
chunks of the reduced grid in worker processes, then the periodic-sinc interpolation and the
normalisation here.  Each pixel's arithmetic does not depend on the chunking, so the result equals
the single-process one.  The workers also return the two smallest eigenvalues of every G(x)
(LAPACK), which the accuracy gate needs.

`gated_errors` is the comparison of Sec. II's identifiability argument made concrete: maps are
compared after per-pixel phase alignment to channel 1, inside the object support eroded by two
pixels, at pixels whose eigen-gap (lambda_2 - lambda_1)/|Lambda| exceeds 1e-3; eigenvalues on
the same reduced pixels.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time

import numpy as np
from scipy import ndimage

from . import pisco_oracle as O

_THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "OPENBLAS_MAIN_FREE")


def make_pool(workers=None):
    """A spawn-started pool of single-threaded workers (spawn: safe after CUDA is initialised)."""
    workers = workers or os.cpu_count() or 1
    saved = {k: os.environ.get(k) for k in _THREAD_VARS}
    for k in _THREAD_VARS:
        os.environ[k] = "1"
    try:
        pool = mp.get_context("spawn").Pool(workers)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return pool, workers


def _pixel_stages(args):
    """G(x), power iteration, low-res images and phase on one chunk of reduced pixels."""
    V_null, lam, Q, xs, v0, iters, calib = args
    L = lam.shape[0]
    G = O.G_direct(V_null, lam, Q, xs)
    v_pi, lam_pi, _ = O.power_iteration(G, v0, iters, L)
    y = O.apodised_lowres(calib, xs)
    v_al = O.phase_align(v_pi, y)
    w = np.linalg.eigvalsh(G)[:, :2] / L
    return v_al, lam_pi, w


def estimate_parallel(calib, grid, tau, shape="ellipsoid", thr=0.05, reduction=1, iters=30, seed=0,
                      pool=None, workers=None):
    """pisco_oracle.estimate (unmasked Gram) with the per-pixel stages spread over `pool`.

    Returns dict(maps [Q][grid], eig [reduced grid], w2 [npix_red, 2] (two smallest eigenvalues
    of G(x)/|Lambda|), k, R, seconds)."""
    t0 = time.perf_counter()
    own = pool is None
    if own:
        pool, workers = make_pool(workers)
    workers = workers or os.cpu_count() or 1
    try:
        calib = np.asarray(calib)
        Q = calib.shape[0]
        grid = tuple(int(g) for g in grid)
        D = len(grid)
        tau = tuple([int(tau)] * D) if np.isscalar(tau) else tuple(tau)
        lam = O.kernel_support(tau, shape)
        red = tuple(g // reduction for g in grid)
        C = O.calibration_matrix(calib, lam, rows="full")
        V_null, U_sig, _ = O.nullspace_svd(C, thr)
        xs = O.grid_points(red)
        v0 = O.start_vectors(seed, xs.shape[0], Q)
        bounds = np.linspace(0, xs.shape[0], min(workers, xs.shape[0]) + 1).astype(int)
        tasks = [(V_null, lam, Q, xs[a:b], v0[a:b], iters, calib) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
        parts = pool.map(_pixel_stages, tasks)
        v_al = np.concatenate([p[0] for p in parts])
        lam_pi = np.concatenate([p[1] for p in parts])
        w2 = np.concatenate([p[2] for p in parts])
        full = O.sinc_interp(v_al, red, grid) if reduction != 1 else v_al
        maps = O.normalize_maps(full)
    finally:
        if own:
            pool.close()
            pool.join()
    return dict(maps=maps.T.reshape((Q,) + grid), eig=lam_pi.reshape(red), w2=w2, k=U_sig.shape[1],
                R=V_null.shape[1], seconds=time.perf_counter() - t0)


def _align(v):
    return v * np.exp(-1j * np.angle(v[:, :1]))


def gate_masks(rho, w2, grid, reduction):
    """(full-grid mask, reduced-grid mask) of the pixels that are compared: inside the object
    support eroded by 2 pixels, with reduced-grid eigen-gap > 1e-3 (a full-grid pixel takes the
    gap of its reduced block)."""
    inner = ndimage.binary_erosion(np.abs(rho) > 0, iterations=2)
    red = tuple(g // reduction for g in grid)
    gap = (w2[:, 1] - w2[:, 0]).reshape(red)
    sl = tuple(slice(None, None, reduction) for _ in grid)
    red_mask = inner[sl] & (gap > 1e-3)
    up = gap
    for ax in range(gap.ndim):
        up = np.repeat(up, reduction, axis=ax)
    return inner & (up > 1e-3), red_mask


def gated_errors(maps, eig, ref, rho, reduction):
    """Map error (relative L2 after channel-1 phase alignment) and max eigenvalue error on the
    gated pixels, for estimator outputs maps [Q][grid] and eig [reduced grid] against a result of
    estimate_parallel."""
    maps = np.asarray(maps)
    Q = maps.shape[0]
    grid = maps.shape[1:]
    full_mask, red_mask = gate_masks(rho, ref["w2"], grid, reduction)
    a = maps.reshape(Q, -1).T
    b = ref["maps"].reshape(Q, -1).T
    fm = full_mask.reshape(-1)
    map_err = float(np.linalg.norm((_align(a) - _align(b))[fm]) / np.linalg.norm(b[fm]))
    rm = red_mask.reshape(-1)
    eig_err = float(np.abs(np.asarray(eig).reshape(-1) - ref["eig"].reshape(-1))[rm].max())
    return dict(map_err=map_err, eig_err=eig_err, pixels=int(fm.sum()), reduced_pixels=int(rm.sum()))
