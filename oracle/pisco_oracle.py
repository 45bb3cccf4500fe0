"""Plain FP64 CPU oracle for the nullspace (ESPIRiT-equivalent) sensitivity-map estimator
with the PISCO accelerations of Lobos, Chan & Haldar (arXiv 2302.13431).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module: only the test
suite, the package's smoke check and the CPU-baseline leg of the benchmark may call it.  It
shares no code with the CUDA path; the only common input is the seeded generator in
`paper_2302_13431_gb300.phantoms`, which holds none of the method's arithmetic.

It follows the naive algorithm of Sec. III-D step by step, in FP64, with the obvious
(slow, memory-hungry) formulation of every object:

  1. the filter support Lambda (Sec. V-B) and the calibration matrix C formed explicitly
     from its definition (Eq. annihil / Eq. C);
  2. the approximate nullspace from an FP64 SVD of C, thresholded at sigma_n < thr*sigma_1
     (Sec. III-B footnote on the threshold);
  3. H(x) per pixel from the filter responses h_r(x,q) (Sec. III-B) and G(x) = H^H H
     (Sec. V-C, first line of Eq. 24);
  4. per-pixel eigensolve of G(x) by a cyclic complex Jacobi method (the exact answer of
     step 4 in Sec. III-D) and, beside it, the simultaneous power iteration of Sec. V-E on
     B(x) = I - G(x)/|Lambda| (Eq. esp_null) from the same start vector the GPU uses;
  5. the smooth phase alpha(x) from a Gaussian-apodised coil-combined low-resolution
     reconstruction (Sec. V-D), periodic-sinc interpolation to the full grid (Sec. V-D),
     and per-pixel unit-norm (sum-of-squares) normalisation (Sec. VI).

Where the paper leaves a detail open this module takes the reading stated in the
function's docstring (Toeplitz orientation of C, unmasked Gram, threshold on singular
values, power-iteration operator/start vector/stop rule, eigenvalue normalisation,
apodisation width, Nyquist split).  The power-iteration start vector generator and the
apodisation width are conventions shared with the CUDA path by definition, not by code:
their parity is unpinned by the paper.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

__all__ = [
    "kernel_support", "difference_set", "calibration_matrix", "nullspace_svd",
    "nullspace_gram_eigh", "filter_response", "G_direct", "jacobi_eigh", "splitmix64", "start_vectors",
    "power_iteration", "apodised_lowres", "phase_align", "sinc_interp_matrix",
    "sinc_interp", "normalize_maps", "estimate", "grid_points",
]

MASK64 = (1 << 64) - 1


# ----------------------------------------------------------------------------------------
# Step 1: filter support and calibration matrix
# ----------------------------------------------------------------------------------------
def kernel_support(tau, shape="ellipsoid"):
    """The FIR support Lambda (Sec. V-B).

    `tau` is a tuple of per-axis radii in (z,)y,x order.  shape="rect" keeps
    ||n||_inf <= tau (the (2 tau+1)^D rectangle); shape="ellipsoid" keeps
    sum_d (n_d/tau_d)^2 <= 1, which for equal radii is the paper's ||n||_2 <= tau.
    Points are returned in lexicographic order with the last (x) coordinate fastest.
    """
    tau = tuple(int(t) for t in tau)
    pts = []
    for n in itertools.product(*[range(-t, t + 1) for t in tau]):
        if shape == "rect":
            pts.append(n)
        elif shape == "ellipsoid":
            if sum((n[d] / tau[d]) ** 2 for d in range(len(tau)) if tau[d] > 0) <= 1.0 + 1e-12 \
                    and all(n[d] == 0 for d in range(len(tau)) if tau[d] == 0):
                pts.append(n)
        else:
            raise ValueError(shape)
    return np.array(pts, dtype=np.int64)


def difference_set(lam):
    """Lambda - Lambda in lexicographic order (x fastest)."""
    diffs = {tuple(a - b) for a in lam for b in lam}
    return np.array(sorted(diffs), dtype=np.int64)


def _box_range(calib_shape):
    """Index range of the centred calibration box: n_d in [-floor(Nc/2), Nc-1-floor(Nc/2)]."""
    return [(-(nc // 2), nc - 1 - nc // 2) for nc in calib_shape]


def calibration_matrix(calib, lam, rows="full"):
    """Explicit calibration matrix C = [C_1 ... C_Q] (Eq. C) built from Eq. annihil:
    row n, column (q, i) holds s_q[n - m_i] (Toeplitz orientation), zero outside the box.

    rows="full": every n whose row can be nonzero (n in box + hull(Lambda)); then
                 C^H C equals the lag table of Sec. V-A with the masking neglected.
    rows="valid": only the n with n - Lambda inside the box (the masked matrix).
    Column index is q*|Lambda| + i.
    """
    calib = np.asarray(calib, dtype=np.complex128)
    Q = calib.shape[0]
    cs = calib.shape[1:]
    D = len(cs)
    lam = np.asarray(lam)
    L = lam.shape[0]
    br = _box_range(cs)
    lo = lam.min(axis=0)
    hi = lam.max(axis=0)
    ranges = [range(br[d][0] + lo[d], br[d][1] + hi[d] + 1) for d in range(D)]
    rows_list = []
    for n in itertools.product(*ranges):
        n = np.array(n)
        if rows == "valid":
            ok = True
            for m in lam:
                k = n - m
                if any(k[d] < br[d][0] or k[d] > br[d][1] for d in range(D)):
                    ok = False
                    break
            if not ok:
                continue
        rows_list.append(n)
    P = len(rows_list)
    C = np.zeros((P, Q * L), dtype=np.complex128)
    off = np.array([nc // 2 for nc in cs])
    for r, n in enumerate(rows_list):
        for i, m in enumerate(lam):
            k = n - m
            if all(br[d][0] <= k[d] <= br[d][1] for d in range(D)):
                idx = tuple(k + off)
                C[r, i::L] = calib[(slice(None),) + idx]
    return C


# ----------------------------------------------------------------------------------------
# Step 2: nullspace by SVD with the sigma_n < thr * sigma_1 rule
# ----------------------------------------------------------------------------------------
def nullspace_svd(C, thr=0.05):
    """FP64 SVD of C; right singular vectors with sigma_n < thr*sigma_1 (strict) form the
    approximate nullspace (Sec. III-A and the threshold footnote of Sec. III-B).  When C has
    fewer rows than columns the missing singular values are zero and their vectors are null.

    Returns (V_null [n x R], U_signal [n x k], sigma [n], ) with columns sorted by
    decreasing singular value.
    """
    n = C.shape[1]
    _, s, Vh = np.linalg.svd(C, full_matrices=True)
    sig = np.zeros(n)
    sig[: s.size] = s
    V = Vh.conj().T
    null = sig < thr * sig[0]
    return V[:, null], V[:, ~null], sig


def nullspace_gram_eigh(C, thr=0.05):
    """The split of nullspace_svd from the FP64 Hermitian eigendecomposition of the Gram C^H C
    (LAPACK) instead of an SVD of C: the eigenvalues are the squared singular values, so
    sigma_n < thr*sigma_1 reads lambda_n < thr^2 lambda_1 (rounding below zero clipped to 0).
    For calibration matrices with many rows (3D: (Nc+2 tau)^3), whose SVD with the full left
    basis is too large.  Returns (V_null, U_signal, sigma) in decreasing order as nullspace_svd.
    """
    A = C.conj().T @ C
    w, V = np.linalg.eigh(0.5 * (A + A.conj().T))
    order = np.argsort(w)[::-1]
    w = np.clip(w[order], 0.0, None)
    V = V[:, order]
    null = w < thr * thr * w[0]
    return V[:, null], V[:, ~null], np.sqrt(w)


# ----------------------------------------------------------------------------------------
# Step 3: filter responses H(x) and G(x) = H^H H
# ----------------------------------------------------------------------------------------
def grid_points(shape):
    """All points of a grid (z,)y,x order, x fastest: x_j = (j - N//2)/N per axis."""
    axes = [(np.arange(n) - n // 2) / n for n in shape]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.reshape(-1) for m in mesh], axis=1)


def filter_response(h, lam, Q, xs):
    """h_r(x,q) = sum_{m in Lambda} h_r[m,q] exp(+i 2 pi m^T x)  (Sec. III-B).

    h: [Q|Lambda| x R] filters (column index q*|Lambda|+i); xs: [npts x D].
    Returns H with shape [npts, R, Q] so that H[j] is the R x Q matrix H(x_j).
    """
    L = lam.shape[0]
    E = np.exp(2j * np.pi * (xs @ lam.T))              # [npts, L]
    hr = h.reshape(Q, L, -1)                            # [Q, L, R]
    return np.einsum("pm,qmr->prq", E, hr)


def G_direct(V_null, lam, Q, xs, chunk=256):
    """G(x) = H(x)^H H(x), i.e. [G]_pq = sum_r conj(h_r(x,p)) h_r(x,q) (Sec. V-C), formed
    pixel by pixel from explicit H(x) (the memory-hungry route the paper starts from)."""
    out = np.empty((xs.shape[0], Q, Q), dtype=np.complex128)
    for s in range(0, xs.shape[0], chunk):
        H = filter_response(V_null, lam, Q, xs[s:s + chunk])
        out[s:s + chunk] = np.einsum("jrp,jrq->jpq", H.conj(), H)
    return out


# ----------------------------------------------------------------------------------------
# Step 4a: exact per-pixel eigensolver (cyclic complex Jacobi)
# ----------------------------------------------------------------------------------------
def jacobi_eigh(G, tol=1e-14, max_sweeps=50):
    """Cyclic Jacobi eigensolver for a batch of Hermitian matrices G[j] (FP64).

    Each rotation annihilates one off-diagonal pair (p,q) of every matrix in the batch at
    once.  Sweeps stop when every off-diagonal Frobenius norm is <= tol*||G||_F.
    Returns (w ascending [npts, Q], V [npts, Q, Q]) with G V = V diag(w).
    """
    A = np.array(G, dtype=np.complex128, copy=True)
    nb, n, _ = A.shape
    V = np.broadcast_to(np.eye(n, dtype=np.complex128), A.shape).copy()
    fro = np.sqrt(np.sum(np.abs(A) ** 2, axis=(1, 2))) + 1e-300
    for _ in range(max_sweeps):
        off = np.sqrt((np.sum(np.abs(A) ** 2, axis=(1, 2))
                       - np.sum(np.abs(np.diagonal(A, axis1=1, axis2=2)) ** 2, axis=1)).clip(0))
        if np.all(off <= tol * fro):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[:, p, q]
                mag = np.abs(apq)
                act = mag > 1e-300
                if not np.any(act):
                    continue
                app = A[:, p, p].real
                aqq = A[:, q, q].real
                # Hermitian 2x2 [[app, apq],[conj(apq), aqq]]: with phase e = apq/|apq| the
                # rotation J = [[c, -s e],[s conj(e), c]] zeroes the (p,q) entry when
                # tan(2 theta) = 2|apq|/(app - aqq); the root with |theta| <= pi/4 is used.
                e = np.where(act, apq / np.where(act, mag, 1.0), 1.0)
                theta = 0.5 * np.arctan2(2 * mag, app - aqq)
                theta = np.where(theta > np.pi / 4, theta - np.pi / 2, theta)
                c = np.cos(theta)
                s = np.sin(theta)
                s = np.where(act, s, 0.0)
                c = np.where(act, c, 1.0)
                # columns: A <- A J
                Ap = A[:, :, p].copy()
                Aq = A[:, :, q].copy()
                A[:, :, p] = c[:, None] * Ap + (s * np.conj(e))[:, None] * Aq
                A[:, :, q] = -(s * e)[:, None] * Ap + c[:, None] * Aq
                # rows: A <- J^H A
                Ap = A[:, p, :].copy()
                Aq = A[:, q, :].copy()
                A[:, p, :] = c[:, None] * Ap + (s * e)[:, None] * Aq
                A[:, q, :] = -(s * np.conj(e))[:, None] * Ap + c[:, None] * Aq
                A[:, p, q] = 0.0
                A[:, q, p] = 0.0
                Vp = V[:, :, p].copy()
                Vq = V[:, :, q].copy()
                V[:, :, p] = c[:, None] * Vp + (s * np.conj(e))[:, None] * Vq
                V[:, :, q] = -(s * e)[:, None] * Vp + c[:, None] * Vq
    w = np.diagonal(A, axis1=1, axis2=2).real
    order = np.argsort(w, axis=1)
    w = np.take_along_axis(w, order, axis=1)
    V = np.take_along_axis(V, order[:, None, :], axis=2)
    return w, V


# ----------------------------------------------------------------------------------------
# Step 4b: simultaneous power iteration (Sec. V-E) on B = I - G/|Lambda| (Eq. esp_null)
# ----------------------------------------------------------------------------------------
def splitmix64(x):
    """SplitMix64 (Steele, Lea & Flood 2014, as published by Vigna): one output for the
    64-bit input counter x, i.e. mix(x + 0x9E3779B97F4A7C15)."""
    z = (int(x) + 0x9E3779B97F4A7C15) & MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
    return z ^ (z >> 31)


def _splitmix64_vec(x):
    x = np.asarray(x, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = x + np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def start_vectors(seed, npix, Q, offset=0):
    """Power-iteration start vectors: v0[j][q] = u(offset+2q) + i u(offset+2q+1) with
    u(t) = ((splitmix64(seed*2^40 + j*2^8 + t) >> 40) - 2^23) / 2^23, a 24-bit uniform in
    [-1, 1).  Exactly representable in FP32, so the CUDA path draws identical vectors.
    offset = 2Q gives the second vector of the block iteration."""
    j = np.arange(npix, dtype=np.uint64)[:, None]
    t = np.arange(offset, offset + 2 * Q, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        ctr = (np.uint64(seed) << np.uint64(40)) + (j << np.uint64(8)) + t
    r = _splitmix64_vec(ctr) >> np.uint64(40)
    u = (r.astype(np.float64) - 2.0 ** 23) / 2.0 ** 23
    return u[:, 0::2] + 1j * u[:, 1::2]


def power_iteration(G, v0, iters, lam_size):
    """Classical power iteration run for all pixels at once (Sec. V-E) on
    B(x) = I - G(x)/|Lambda| (Eq. esp_null), whose dominant eigenvector is the eigenvector
    of G(x) with the smallest eigenvalue.  Each step: v <- B v, v <- v/||v||.  After `iters`
    steps returns v, lambda = Re(v^H G v)/|Lambda| and the residual
    ||G v - lambda |Lambda| v|| / |Lambda|.
    """
    v = np.array(v0, dtype=np.complex128)
    v = v / np.linalg.norm(v, axis=1, keepdims=True)
    for _ in range(iters):
        Gv = np.einsum("jpq,jq->jp", G, v)
        v = v - Gv / lam_size
        v = v / np.linalg.norm(v, axis=1, keepdims=True)
    Gv = np.einsum("jpq,jq->jp", G, v)
    lam = np.real(np.sum(np.conj(v) * Gv, axis=1)) / lam_size
    res = np.linalg.norm(Gv - (lam * lam_size)[:, None] * v, axis=1) / lam_size
    return v, lam, res


def block_power_iteration(G, V0, iters, lam_size):
    """Power iteration on a two-vector block (subspace iteration) for pixels whose two smallest
    eigenvalues of G(x) are close, then Rayleigh-Ritz on the block.  Each step applies
    B = I - G/|Lambda| to both vectors and re-orthonormalises them by Gram-Schmidt (first
    vector normalised, second made orthogonal to it and normalised).  At the end the 2x2 matrix
    H = V^H G V is diagonalised and the Ritz vector of its smallest eigenvalue is returned with
    lambda = that eigenvalue / |Lambda|.  V0: [npix, Q, 2]."""
    V = np.array(V0, dtype=np.complex128)
    def orth(V):
        v1 = V[:, :, 0] / np.linalg.norm(V[:, :, 0], axis=1, keepdims=True)
        w2 = V[:, :, 1] - np.sum(np.conj(v1) * V[:, :, 1], axis=1, keepdims=True) * v1
        v2 = w2 / np.linalg.norm(w2, axis=1, keepdims=True)
        return np.stack([v1, v2], axis=2)
    V = orth(V)
    for _ in range(iters):
        GV = np.einsum("jpq,jqb->jpb", G, V)
        V = orth(V - GV / lam_size)
    GV = np.einsum("jpq,jqb->jpb", G, V)
    H = np.einsum("jpa,jpb->jab", np.conj(V), GV)
    H = 0.5 * (H + np.conj(np.swapaxes(H, 1, 2)))
    w, Y = np.linalg.eigh(H)
    v = np.einsum("jqb,jb->jq", V, Y[:, :, 0])
    v = v / np.linalg.norm(v, axis=1, keepdims=True)
    return v, w[:, 0] / lam_size


# ----------------------------------------------------------------------------------------
# Step 5: smooth phase, periodic-sinc interpolation, normalisation
# ----------------------------------------------------------------------------------------
def apodised_lowres(calib, xs):
    """Coil images of the Gaussian-apodised calibration data evaluated at xs (Sec. V-D):
    y_q(x) = sum_n a[n] s_q[n] exp(+i 2 pi n^T x), a[n] = prod_d exp(-(n_d/(Nc_d/4))^2/2).
    Returns [npts, Q]."""
    calib = np.asarray(calib, dtype=np.complex128)
    Q = calib.shape[0]
    cs = calib.shape[1:]
    axes = [np.arange(nc) - nc // 2 for nc in cs]
    mesh = np.meshgrid(*axes, indexing="ij")
    n = np.stack([m.reshape(-1) for m in mesh], axis=1)            # [Nc^D, D]
    a = np.ones(n.shape[0])
    for d, nc in enumerate(cs):
        a = a * np.exp(-0.5 * (n[:, d] / (nc / 4.0)) ** 2)
    s = calib.reshape(Q, -1) * a[None, :]
    E = np.exp(2j * np.pi * (xs @ n.T))                              # [npts, Nc^D]
    return E @ s.T


def phase_align(v, y):
    """Choose alpha(x) so that the coil-combined low-res reconstruction v^H y becomes real
    and non-negative (Sec. V-D): v <- v * rho/|rho| with rho = sum_q conj(v_q) y_q.  Pixels
    with rho == 0 are left unchanged."""
    rho = np.sum(np.conj(v) * y, axis=1)
    mag = np.abs(rho)
    ph = np.where(mag > 0, rho / np.where(mag > 0, mag, 1.0), 1.0)
    return v * ph[:, None]


def sinc_interp_matrix(n_in, n_out):
    """Periodic-sinc interpolation along one axis (Sec. V-D) as an explicit n_out x n_in
    matrix: DFT of the coarse samples at x_j = (j - n_in//2)/n_in, keep the band
    k in [-n_in/2, n_in/2 - 1] (for even n_in the Nyquist coefficient is split equally
    between +-n_in/2), evaluate the trigonometric polynomial at x_i = (i - n_out//2)/n_out."""
    xj = (np.arange(n_in) - n_in // 2) / n_in
    xi = (np.arange(n_out) - n_out // 2) / n_out
    ks = np.arange(-(n_in // 2), n_in - n_in // 2)
    F = np.exp(-2j * np.pi * np.outer(ks, xj)) / n_in                # [n_in(k), n_in(j)]
    Ein = np.exp(2j * np.pi * np.outer(xi, ks))                        # [n_out, k]
    if n_in % 2 == 0 and n_out != n_in:
        nyq = 0  # index of k = -n_in/2
        Ein[:, nyq] = 0.5 * (np.exp(-1j * np.pi * n_in * xi) + np.exp(1j * np.pi * n_in * xi))
    return Ein @ F


def sinc_interp(vr, in_shape, out_shape):
    """Separable periodic-sinc interpolation of [npts_in, Q] samples on `in_shape` to
    `out_shape` (both (z,)y,x).  Returns [npts_out, Q]."""
    Q = vr.shape[1]
    arr = vr.T.reshape((Q,) + tuple(in_shape))
    for d in range(len(in_shape)):
        M = sinc_interp_matrix(in_shape[d], out_shape[d])
        arr = np.moveaxis(np.tensordot(M, arr, axes=([1], [d + 1])), 0, d + 1)
    return arr.reshape(Q, -1).T


def normalize_maps(c):
    """Sum-of-squares (unit 2-norm per pixel) normalisation (Sec. VI); zero pixels stay 0."""
    nrm = np.linalg.norm(c, axis=1, keepdims=True)
    return np.where(nrm > 0, c / np.where(nrm > 0, nrm, 1.0), 0.0)


# ----------------------------------------------------------------------------------------
# The whole naive pipeline + PISCO reduced grid, as the CUDA path computes it
# ----------------------------------------------------------------------------------------
def estimate(calib, grid, tau, shape="ellipsoid", thr=0.05, reduction=1, iters=30, seed=0,
             rows="full", exact=True, return_all=False):
    """Sensitivity maps and eigenvalue map for one calibration block.

    calib: complex [Q][Nc...] (z,y,x);  grid: full image grid;  tau: per-axis radius;
    reduction: grid-reduction factor f (reduced grid = grid/f, Sec. V-D);  iters: power
    iterations.  Returns maps [Q][grid...] (complex128, unit norm per pixel) and the
    eigenvalue map lambda_min(G)/|Lambda| on the reduced grid (from power iteration), plus
    every intermediate when return_all is set.
    """
    calib = np.asarray(calib)
    Q = calib.shape[0]
    grid = tuple(int(g) for g in grid)
    D = len(grid)
    tau = tuple([int(tau)] * D) if np.isscalar(tau) else tuple(tau)
    lam = kernel_support(tau, shape)
    L = lam.shape[0]
    red = tuple(g // reduction for g in grid)
    C = calibration_matrix(calib, lam, rows=rows)
    V_null, U_sig, sig = nullspace_svd(C, thr)
    xs = grid_points(red)
    G = G_direct(V_null, lam, Q, xs)
    v0 = start_vectors(seed, xs.shape[0], Q)
    v_pi, lam_pi, res = power_iteration(G, v0, iters, L)
    y = apodised_lowres(calib, xs)
    v_al = phase_align(v_pi, y)
    full = sinc_interp(v_al, red, grid) if reduction != 1 else v_al
    maps = normalize_maps(full)
    out = dict(maps=maps.T.reshape((Q,) + grid), eig=lam_pi.reshape(red))
    if return_all:
        out.update(lam=lam, C=C, V_null=V_null, U_sig=U_sig, sigma=sig, xs=xs, G=G, v0=v0,
                   v_pi=v_pi, res=res, y=y, v_aligned=v_al, R=V_null.shape[1],
                   k=U_sig.shape[1])
        if exact:
            w, V = jacobi_eigh(G)
            v_ex = phase_align(V[:, :, 0], y)
            out.update(w_exact=w, v_exact=v_ex, eig_exact=(w[:, 0] / L).reshape(red))
    return out
