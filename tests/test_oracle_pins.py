"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Every test here checks the oracle against something other than itself: a library routine
(LAPACK through numpy, scipy's convolution, numpy's FFT), a closed form, an identity the
paper states, a published test vector, or brute force on tiny inputs.  None needs a GPU.
"""
import os

import numpy as np
import pytest
from scipy import signal

from oracle import pisco_oracle as O
from paper_2302_13431_gb300.phantoms import make_case, centered_dft, crop_center, grid_coords

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _rand_calib(rng, Q, shape):
    return (rng.standard_normal((Q,) + shape) + 1j * rng.standard_normal((Q,) + shape))


# ---------------------------------------------------------------------------------------
# Lambda (Sec. V-B)
# ---------------------------------------------------------------------------------------
def test_support_counts_match_lattice_point_counts():
    """|Lambda| equals the number of lattice points in the disc/ball (OEIS A000328,
    A000605) or the (2 tau + 1)^D rectangle."""
    with open(os.path.join(GOLD, "lattice_counts.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for kind, nd, r, cnt in rows:
        lam = O.kernel_support((int(r),) * int(nd), kind)
        assert lam.shape[0] == int(cnt), (kind, nd, r)
        if kind == "ellipsoid":
            assert np.all(np.sum(lam ** 2, axis=1) <= int(r) ** 2)
        assert len({tuple(p) for p in lam}) == lam.shape[0]


def test_support_order_is_lexicographic_x_fastest():
    lam = O.kernel_support((1, 1), "rect")
    assert [tuple(p) for p in lam] == sorted(tuple(p) for p in lam)
    assert tuple(lam[1]) == (-1, 0)


def test_difference_set_brute_force():
    lam = O.kernel_support((3, 3), "ellipsoid")
    D = O.difference_set(lam)
    brute = set()
    for a in lam:
        for b in lam:
            brute.add((a[0] - b[0], a[1] - b[1]))
    assert len(D) == len(brute)
    assert {tuple(d) for d in D} == brute
    assert np.all(np.abs(D) <= 6)


# ---------------------------------------------------------------------------------------
# C (Eq. annihil, Eq. C) and the FFT Gram of Sec. V-A
# ---------------------------------------------------------------------------------------
def test_calibration_matrix_applies_the_annihilation_convolution():
    """C h must equal sum_q (h_q * s_q)[n] (Eq. annihil) for every row n of the full
    matrix; scipy's 2D convolution is the independent route."""
    rng = np.random.default_rng(1)
    Q, cs, tau = 3, (7, 6), (2, 1)
    s = _rand_calib(rng, Q, cs)
    lam = O.kernel_support(tau, "rect")
    C = O.calibration_matrix(s, lam, rows="full")
    h = rng.standard_normal(Q * lam.shape[0]) + 1j * rng.standard_normal(Q * lam.shape[0])
    conv = 0
    for q in range(Q):
        ker = np.zeros((2 * tau[0] + 1, 2 * tau[1] + 1), complex)
        for i, m in enumerate(lam):
            ker[m[0] + tau[0], m[1] + tau[1]] = h[q * lam.shape[0] + i]
        conv = conv + signal.convolve2d(s[q], ker, mode="full")
    assert C.shape[0] == conv.size
    np.testing.assert_allclose(C @ h, conv.reshape(-1), rtol=0, atol=1e-12)


def test_valid_rows_are_the_masked_rows():
    rng = np.random.default_rng(2)
    s = _rand_calib(rng, 2, (9, 8))
    lam = O.kernel_support((2, 2), "rect")
    Cv = O.calibration_matrix(s, lam, rows="valid")
    assert Cv.shape[0] == (9 - 4) * (8 - 4)
    # valid convolution through scipy
    h = rng.standard_normal(2 * 25) + 1j * rng.standard_normal(2 * 25)
    conv = 0
    for q in range(2):
        ker = np.zeros((5, 5), complex)
        for i, m in enumerate(lam):
            ker[m[0] + 2, m[1] + 2] = h[q * 25 + i]
        conv = conv + signal.convolve2d(s[q], ker, mode="valid")
    np.testing.assert_allclose(Cv @ h, conv.reshape(-1), atol=1e-12)


def _fft_lags(s, lags, Lpad):
    """Sec. V-A: zero-padded FFTs of every channel, products conj(S_p) S_q and inverse
    FFTs, read at the lags.  Written here independently of the oracle."""
    Q = s.shape[0]
    cs = s.shape[1:]
    pad = np.zeros((Q,) + (Lpad,) * len(cs), complex)
    for idx in np.ndindex(*cs):
        n = tuple((i - nc // 2) % Lpad for i, nc in zip(idx, cs))
        pad[(slice(None),) + n] = s[(slice(None),) + idx]
    S = np.fft.fftn(pad, axes=tuple(range(1, len(cs) + 1)))
    R = np.empty((Q, Q, len(lags)), complex)
    for p in range(Q):
        for q in range(Q):
            r = np.fft.ifftn(np.conj(S[p]) * S[q])
            for t, d in enumerate(lags):
                R[p, q, t] = r[tuple(int(di) % Lpad for di in d)]
    return R


@pytest.mark.parametrize("ndim", [2, 3])
def test_fft_gram_equals_full_CtC(ndim):
    """Masking neglected, the FFT route of Sec. V-A gives exactly C_full^H C_full; the
    result does not depend on the padded length L >= Nc + 2 tau."""
    rng = np.random.default_rng(3)
    Q = 3
    cs = (6, 7) if ndim == 2 else (5, 4, 6)
    tau = (2,) * ndim if ndim == 2 else (1, 1, 1)
    lam = O.kernel_support(tau, "ellipsoid")
    s = _rand_calib(rng, Q, cs)
    C = O.calibration_matrix(s, lam, rows="full")
    A = C.conj().T @ C
    lags = O.difference_set(lam)
    lag_index = {tuple(d): t for t, d in enumerate(lags)}
    for Lpad in (max(cs) + 2 * max(tau), 16):
        R = _fft_lags(s, lags, Lpad)
        L = lam.shape[0]
        B = np.empty_like(A)
        for p in range(Q):
            for q in range(Q):
                for i in range(L):
                    for j in range(L):
                        B[p * L + i, q * L + j] = R[p, q, lag_index[tuple(lam[i] - lam[j])]]
        np.testing.assert_allclose(B, A, rtol=0, atol=1e-11 * np.abs(A).max())


# ---------------------------------------------------------------------------------------
# Nullspace (Sec. III-A, threshold footnote)
# ---------------------------------------------------------------------------------------
def test_nullspace_svd_matches_lapack_eigh_of_gram():
    case = make_case((48, 48), 4, (16, 16), seed=5, phase="linear")
    lam = O.kernel_support((2, 2), "ellipsoid")
    C = O.calibration_matrix(case.calib, lam, rows="full")
    Vn, Us, sig = O.nullspace_svd(C, 0.05)
    w, U = np.linalg.eigh(C.conj().T @ C)
    keep = w >= 0.05 ** 2 * w.max()
    assert keep.sum() == Us.shape[1]
    P1 = Us @ Us.conj().T
    P2 = U[:, keep] @ U[:, keep].conj().T
    np.testing.assert_allclose(P1, P2, atol=1e-9)
    W = Vn @ Vn.conj().T
    np.testing.assert_allclose(W @ W, W, atol=1e-12)
    assert abs(np.trace(W).real - Vn.shape[1]) < 1e-10
    np.testing.assert_allclose(Vn.conj().T @ Vn, np.eye(Vn.shape[1]), atol=1e-12)
    assert np.all(sig[:-1] >= sig[1:])


@pytest.mark.parametrize("grid, Q, cs, tau", [((48, 48), 4, (16, 16), (2, 2)), ((12, 16, 12), 3, (8, 10, 8), (1, 2, 1))])
def test_gram_eigh_route_equals_the_svd_route(grid, Q, cs, tau):
    """nullspace_gram_eigh (eigendecomposition of C^H C) gives the SVD route's split: same k,
    same signal projector, orthonormal null basis, singular values equal."""
    case = make_case(grid, Q, cs, seed=9, phase="poly4")
    lam = O.kernel_support(tau, "ellipsoid")
    C = O.calibration_matrix(case.calib, lam, rows="full")
    Vn, Us, sig = O.nullspace_svd(C, 0.05)
    Vn2, Us2, sig2 = O.nullspace_gram_eigh(C, 0.05)
    assert Us2.shape[1] == Us.shape[1] and Vn2.shape[1] == Vn.shape[1]
    np.testing.assert_allclose(Us2 @ Us2.conj().T, Us @ Us.conj().T, atol=1e-9)
    np.testing.assert_allclose(Vn2.conj().T @ Vn2, np.eye(Vn2.shape[1]), atol=1e-12)
    k = Us.shape[1]
    np.testing.assert_allclose(sig2[:k], sig[:k], rtol=1e-9)
    # a threshold placed between two singular values moves the split by exactly one
    thr = 0.5 * (sig[k - 1] + sig[k - 2]) / sig[0]
    assert O.nullspace_gram_eigh(C, thr)[1].shape[1] == O.nullspace_svd(C, thr)[1].shape[1] == k - 1


def test_threshold_is_strict_and_counts_missing_singular_values():
    # P < n: C has 2 rows and 4 columns -> at least 2 exactly-null directions
    C = np.array([[1.0, 0, 0, 0], [0, 0.05, 0, 0]], complex)
    Vn, Us, sig = O.nullspace_svd(C, 0.05)
    # sigma_2 = 0.05 * sigma_1 is NOT below the strict threshold -> signal
    assert Us.shape[1] == 2 and Vn.shape[1] == 2
    np.testing.assert_allclose(sig, [1.0, 0.05, 0, 0])


def _bandlimited_case(N=48, Q=3, Nc=20, seed=11):
    """Noise-free data whose maps are exact trigonometric polynomials on Lambda_c =
    {||k||_inf <= 1}: the cross-relation filters of Eq. f2 then annihilate the data."""
    rng = np.random.default_rng(seed)
    ys, xs = np.meshgrid(*grid_coords((N, N)), indexing="ij")
    lam_c = O.kernel_support((1, 1), "rect")
    coef = rng.standard_normal((Q, len(lam_c))) + 1j * rng.standard_normal((Q, len(lam_c)))
    coef[:, 4] += 4.0  # strong DC so the maps do not vanish
    maps = np.zeros((Q, N, N), complex)
    for q in range(Q):
        for i, m in enumerate(lam_c):
            maps[q] += coef[q, i] * np.exp(2j * np.pi * (m[0] * ys + m[1] * xs))
    rho = np.zeros((N, N), complex)
    rho[(xs / 0.3) ** 2 + (ys / 0.2) ** 2 <= 1] = 1.0
    rho[((xs - 0.05) / 0.1) ** 2 + (ys / 0.08) ** 2 <= 1] += 0.5j
    k = centered_dft(maps * rho[None], (1, 2))
    return crop_center(k, (Nc, Nc)), coef, lam_c


def test_cross_relation_filters_lie_in_the_nullspace():
    """Eq. f2: h = (-c_j on channel i, c_i on channel j) annihilates noise-free data with
    maps bandlimited to Lambda_c subset Lambda, so it must lie in the thresholded
    nullspace of the masked C."""
    calib, coef, lam_c = _bandlimited_case()
    lam = O.kernel_support((2, 2), "rect")
    Cv = O.calibration_matrix(calib, lam, rows="valid")
    Vn, Us, _ = O.nullspace_svd(Cv, 0.05)
    L = lam.shape[0]
    pos = {tuple(m): i for i, m in enumerate(lam)}
    for (i, j) in [(0, 1), (0, 2), (1, 2)]:
        h = np.zeros(3 * L, complex)
        for t, m in enumerate(lam_c):
            h[i * L + pos[tuple(m)]] = -coef[j, t]
            h[j * L + pos[tuple(m)]] = coef[i, t]
        h /= np.linalg.norm(h)
        assert np.linalg.norm(Cv @ h) < 1e-9 * np.linalg.norm(Cv)
        assert np.linalg.norm(Us.conj().T @ h) < 1e-9


# ---------------------------------------------------------------------------------------
# G(x) (Sec. V-C, Eq. 24, Eq. esp_null)
# ---------------------------------------------------------------------------------------
def _random_split(rng, n, R):
    M = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    U, _ = np.linalg.qr(M)
    return U[:, :R], U[:, R:]


def test_G_three_routes_agree_and_espirit_identity():
    rng = np.random.default_rng(7)
    Q = 3
    lam = O.kernel_support((2, 2), "ellipsoid")
    L = lam.shape[0]
    n = Q * L
    Vn, Us = _random_split(rng, n, 25)
    xs = O.grid_points((9, 8))
    G = O.G_direct(Vn, lam, Q, xs)
    # Eq. 24 double sum through W = sum_r h_r h_r^H
    W = Vn @ Vn.conj().T
    E = np.exp(2j * np.pi * (xs @ lam.T))           # e^{i2pi n_s x}
    G2 = np.empty_like(G)
    for p in range(Q):
        for q in range(Q):
            Wqp = W[q * L:(q + 1) * L, p * L:(p + 1) * L]   # [s, t]
            G2[:, p, q] = np.einsum("js,st,jt->j", E, Wqp, E.conj())
    np.testing.assert_allclose(G2, G, atol=1e-12)
    # collapsed kernel K_pq[d] = sum_{n_s - m_t = d} W_qp[s,t]
    lags = O.difference_set(lam)
    li = {tuple(d): t for t, d in enumerate(lags)}
    K = np.zeros((Q, Q, len(lags)), complex)
    for p in range(Q):
        for q in range(Q):
            for s_ in range(L):
                for t in range(L):
                    K[p, q, li[tuple(lam[s_] - lam[t])]] += W[q * L + s_, p * L + t]
    G3 = np.einsum("jd,pqd->jpq", np.exp(2j * np.pi * (xs @ lags.T)), K)
    np.testing.assert_allclose(G3, G, atol=1e-12)
    # Eq. esp_null: I - G/|Lambda| = H_s^H H_s / |Lambda| for the complementary basis
    Hs = O.filter_response(Us, lam, Q, xs)
    Bs = np.einsum("jrp,jrq->jpq", Hs.conj(), Hs)
    np.testing.assert_allclose(L * np.eye(Q)[None] - G, Bs, atol=1e-11)
    w = np.linalg.eigvalsh(G)
    assert w.min() > -1e-10 and w.max() < L + 1e-10


def test_mean_trace_of_G_equals_R():
    """Averaging tr G(x) over a grid with N_r > 2 tau keeps only the zero lag:
    mean tr G = tr W = R."""
    rng = np.random.default_rng(8)
    Q = 2
    lam = O.kernel_support((3, 3), "ellipsoid")
    Vn, _ = _random_split(rng, Q * lam.shape[0], 31)
    G = O.G_direct(Vn, lam, Q, O.grid_points((7, 10)))
    assert abs(np.mean(np.trace(G, axis1=1, axis2=2)).real - 31) < 1e-10


def test_filter_response_brute_force():
    rng = np.random.default_rng(9)
    lam = O.kernel_support((1, 1), "rect")
    h = rng.standard_normal((2 * 9, 2)) + 1j * rng.standard_normal((2 * 9, 2))
    x = np.array([[0.1, -0.3]])
    H = O.filter_response(h, lam, 2, x)
    for r in range(2):
        for q in range(2):
            val = sum(h[q * 9 + i, r] * np.exp(2j * np.pi * (m[0] * x[0, 0] + m[1] * x[0, 1]))
                      for i, m in enumerate(lam))
            assert abs(H[0, r, q] - val) < 1e-13


# ---------------------------------------------------------------------------------------
# Eigensolvers (Sec. III-D step 4, Sec. V-E)
# ---------------------------------------------------------------------------------------
def test_jacobi_matches_lapack():
    rng = np.random.default_rng(10)
    A = rng.standard_normal((40, 7, 7)) + 1j * rng.standard_normal((40, 7, 7))
    A = A + A.conj().transpose(0, 2, 1)
    w, V = O.jacobi_eigh(A)
    np.testing.assert_allclose(w, np.linalg.eigvalsh(A), atol=1e-12)
    np.testing.assert_allclose(np.einsum("jpq,jqk->jpk", A, V), V * w[:, None, :], atol=1e-11)
    np.testing.assert_allclose(np.einsum("jqp,jqk->jpk", V.conj(), V), np.broadcast_to(np.eye(7), A.shape), atol=1e-12)


def test_power_iteration_closed_form_2x2():
    """G = diag(0, |Lambda|/2): B = diag(1, 1/2), so from v0 = (1,1) the iterate after t
    steps is (1, 2^-t)/||.||; lambda = 2^-2t/(1+2^-2t)/2."""
    L = 10.0
    G = np.array([[[0, 0], [0, L / 2]]], complex)
    for t in (0, 1, 5):
        v, lam, res = O.power_iteration(G, np.array([[1.0, 1.0]]), t, L)
        ref = np.array([1.0, 2.0 ** -t]) / np.hypot(1.0, 2.0 ** -t)
        np.testing.assert_allclose(np.abs(v[0]), ref, atol=1e-15)
        assert abs(lam[0] - 0.5 * 4.0 ** -t / (1 + 4.0 ** -t)) < 1e-15


def test_power_iteration_converges_to_jacobi_on_gapped_pixels():
    rng = np.random.default_rng(12)
    Q, L = 5, 13.0
    U, _ = np.linalg.qr(rng.standard_normal((30, Q, Q)) + 1j * rng.standard_normal((30, Q, Q)))
    ev = np.sort(rng.uniform(0.3, 1.0, (30, Q)), axis=1) * L
    ev[:, 0] = rng.uniform(0, 0.01, 30) * L
    G = np.einsum("jpk,jk,jqk->jpq", U, ev, U.conj())
    v, lam, res = O.power_iteration(G, O.start_vectors(3, 30, Q), 200, L)
    w, V = O.jacobi_eigh(G)
    ph = np.sum(np.conj(V[:, :, 0]) * v, axis=1)
    np.testing.assert_allclose(np.abs(ph), 1.0, atol=1e-10)
    np.testing.assert_allclose(lam, w[:, 0] / L, atol=1e-12)
    assert res.max() < 1e-10


def test_splitmix64_published_vectors():
    vals = [int(l) for l in open(os.path.join(GOLD, "splitmix64_vectors.txt")) if l.strip() and not l.startswith("#")]
    state = vals[0]
    gamma = 0x9E3779B97F4A7C15
    for i, want in enumerate(vals[1:]):
        assert O.splitmix64(state + i * gamma) == want
    # the vectorised form agrees with the scalar one
    ctr = np.array([state + i * gamma for i in range(5)], dtype=object)
    vec = O._splitmix64_vec(np.array([int(c) & O.MASK64 for c in ctr], dtype=np.uint64))
    assert [int(x) for x in vec] == vals[1:]


def test_start_vectors_are_fp32_exact_and_uniform():
    v = O.start_vectors(7, 1000, 8)
    assert np.all(v.real.astype(np.float32) == v.real)
    assert np.all(np.abs(v.real) <= 1) and np.all(np.abs(v.imag) <= 1)
    assert abs(np.mean(v.real)) < 0.03 and abs(np.var(v.real) - 1 / 3) < 0.02
    assert not np.allclose(O.start_vectors(8, 10, 8), v[:10])


# ---------------------------------------------------------------------------------------
# Phase, interpolation, normalisation (Sec. V-D, Sec. VI)
# ---------------------------------------------------------------------------------------
def test_apodised_lowres_matches_inverse_fft():
    """y_q(x) on the N grid equals the inverse DFT of the apodised, zero-padded box."""
    rng = np.random.default_rng(13)
    s = _rand_calib(rng, 2, (6, 8))
    N = 16
    y = O.apodised_lowres(s, O.grid_points((N, N)))
    a = np.outer(np.exp(-0.5 * ((np.arange(6) - 3) / 1.5) ** 2), np.exp(-0.5 * ((np.arange(8) - 4) / 2.0) ** 2))
    full = np.zeros((2, N, N), complex)
    full[:, N // 2 - 3:N // 2 + 3, N // 2 - 4:N // 2 + 4] = s * a
    img = np.fft.fftshift(np.fft.ifftn(np.fft.ifftshift(full, axes=(1, 2)), axes=(1, 2)), axes=(1, 2)) * N * N
    np.testing.assert_allclose(y.T.reshape(2, N, N), img, atol=1e-10)


def test_phase_align_invariance_and_realness():
    rng = np.random.default_rng(14)
    v = rng.standard_normal((50, 4)) + 1j * rng.standard_normal((50, 4))
    y = rng.standard_normal((50, 4)) + 1j * rng.standard_normal((50, 4))
    a = O.phase_align(v, y)
    b = O.phase_align(v * np.exp(1j * rng.uniform(0, 6.3, (50, 1))), y)
    np.testing.assert_allclose(a, b, atol=1e-13)
    comb = np.sum(np.conj(a) * y, axis=1)
    assert np.all(np.abs(comb.imag) < 1e-12) and np.all(comb.real >= 0)
    z = O.phase_align(v, np.zeros_like(y))
    np.testing.assert_array_equal(z, v)


@pytest.mark.parametrize("nin,nout", [(8, 32), (9, 27), (16, 16), (6, 24)])
def test_sinc_interp_exact_on_band_limited_trig_polynomials(nin, nout):
    rng = np.random.default_rng(15)
    ks = np.arange(-(nin // 2) + (1 if nin % 2 == 0 else 0), nin - nin // 2)
    c = rng.standard_normal(len(ks)) + 1j * rng.standard_normal(len(ks))
    f = lambda x: np.exp(2j * np.pi * np.outer(x, ks)) @ c
    xin = (np.arange(nin) - nin // 2) / nin
    xout = (np.arange(nout) - nout // 2) / nout
    M = O.sinc_interp_matrix(nin, nout)
    np.testing.assert_allclose(M @ f(xin), f(xout), atol=1e-11)
    if nout % nin == 0:
        fct = nout // nin
        # coarse point j sits at fine index f*j + (nout//2 - f*(nin//2))
        idx = fct * np.arange(nin) + (nout // 2 - fct * (nin // 2))
        np.testing.assert_allclose((M @ f(xin))[idx], f(xin), atol=1e-11)
        # coarse samples of any signal are reproduced (interpolation property)
        g = rng.standard_normal(nin)
        np.testing.assert_allclose((M @ g)[idx], g, atol=1e-11)
    if nin == nout:
        np.testing.assert_allclose(M, np.eye(nin), atol=1e-12)


def test_sinc_interp_nyquist_split_keeps_real_signals_real():
    g = np.random.default_rng(16).standard_normal(8)
    out = O.sinc_interp_matrix(8, 32) @ g
    assert np.abs(out.imag).max() < 1e-12


def test_sinc_interp_separable_2d():
    rng = np.random.default_rng(17)
    v = rng.standard_normal((6 * 4, 2)) + 0j
    out = O.sinc_interp(v, (6, 4), (12, 16))
    My, Mx = O.sinc_interp_matrix(6, 12), O.sinc_interp_matrix(4, 16)
    ref = np.einsum("ya,xb,qab->qyx", My, Mx, v.T.reshape(2, 6, 4)).reshape(2, -1).T
    np.testing.assert_allclose(out, ref, atol=1e-12)


def test_normalize_maps():
    c = np.array([[3.0, 4.0], [0.0, 0.0]], complex)
    n = O.normalize_maps(c)
    np.testing.assert_allclose(n, [[0.6, 0.8], [0, 0]])


# ---------------------------------------------------------------------------------------
# End to end (Sec. III-B rank claim, Fig. sv_H)
# ---------------------------------------------------------------------------------------
def test_end_to_end_small_case_support_and_maps():
    """Inside the support lambda_min(G)/|Lambda| is ~0 and well outside it is clearly
    positive (Sec. III-B rank claim, Fig. sv_H); power iteration agrees with the Jacobi
    eigenvector inside; the estimated maps are close to the true ones after channel-1
    phase alignment; every output pixel has unit norm."""
    from scipy import ndimage
    case = make_case((32, 32), 4, (16, 16), seed=1, phase="linear", noise=0.0)
    out = O.estimate(case.calib, (32, 32), 2, shape="rect", reduction=1, iters=60,
                     return_all=True, exact=True)
    supp = np.abs(case.rho) > 0
    inner = ndimage.binary_erosion(supp, iterations=2)
    far = ~ndimage.binary_dilation(supp, iterations=2)
    e = out["eig"]
    assert np.median(e[inner]) < 3e-3
    assert np.median(e[far]) > 0.3 and e[far].min() > 0.05
    m = inner.reshape(-1)
    vp, ve = out["v_aligned"][m], out["v_exact"][m]
    assert np.linalg.norm(vp - ve) / np.linalg.norm(ve) < 1e-8
    al = lambda v: v * np.exp(-1j * np.angle(v[:, :1]))
    mt = case.maps.reshape(4, -1).T[m]
    me = out["maps"].reshape(4, -1).T[m]
    assert np.linalg.norm(al(mt) - al(me)) / np.linalg.norm(mt) < 0.05
    assert np.allclose(np.linalg.norm(out["maps"].reshape(4, -1), axis=0), 1.0)


def _hermitian_with_spectrum(rng, Q, lams):
    M = rng.standard_normal((Q, Q)) + 1j * rng.standard_normal((Q, Q))
    U, _ = np.linalg.qr(M)
    return (U * np.asarray(lams)) @ U.conj().T, U


def test_block_power_iteration_spans_the_matrix_power_subspace():
    """After t steps the block spans (I - G/L)^t V0: compared through the projectors, with the
    power formed explicitly (matrix_power) and orthonormalised by QR."""
    rng = np.random.default_rng(31)
    Q, L, t = 6, 9.0, 5
    G, _ = _hermitian_with_spectrum(rng, Q, [0.1, 0.4, 2.0, 3.0, 5.0, 8.0])
    V0 = rng.standard_normal((1, Q, 2)) + 1j * rng.standard_normal((1, Q, 2))
    Bt = np.linalg.matrix_power(np.eye(Q) - G / L, t)
    Qm, _ = np.linalg.qr(Bt @ V0[0])
    P_ref = Qm @ Qm.conj().T
    # the oracle's block before Rayleigh-Ritz is recovered from its Ritz vector's subspace:
    # run with t steps and check the Ritz vector lies in span(Bt V0)
    v, lam = O.block_power_iteration(G[None], V0, t, L)
    assert np.linalg.norm(P_ref @ v[0] - v[0]) < 1e-12
    # and it is the Ritz vector of the projected matrix
    H = Qm.conj().T @ G @ Qm
    w, Y = np.linalg.eigh(H)
    assert abs(lam[0] - w[0] / L) < 1e-12
    y = Qm @ Y[:, 0]
    assert abs(abs(np.vdot(y, v[0])) - 1.0) < 1e-12


def test_block_iteration_converges_where_single_vector_iteration_lags():
    """Two nearly equal smallest eigenvalues (gap 1e-3 |Lambda|) and a large third one: after 30
    steps the single-vector iteration is still far from the null vector (its rate is set by
    lambda_2), the block iteration with Rayleigh-Ritz has converged at the rate set by lambda_3:
    1 - |<v, v*>| ~ ((1 - lambda_3/L) / (1 - lambda_1/L))^(2t) = 0.7^60 = 5e-10."""
    rng = np.random.default_rng(32)
    Q, L = 8, 20.0
    G, U = _hermitian_with_spectrum(rng, Q, [0.0, 0.02, 6.0, 7.0, 9.0, 11.0, 14.0, 19.0])
    v0 = O.start_vectors(3, 1, Q)
    V0 = np.stack([v0, O.start_vectors(3, 1, Q, offset=2 * Q)], axis=2)
    vp, _, _ = O.power_iteration(G[None], v0, 30, L)
    vb, lb = O.block_power_iteration(G[None], V0, 30, L)
    err_p = 1 - abs(np.vdot(U[:, 0], vp[0]))
    err_b = 1 - abs(np.vdot(U[:, 0], vb[0]))
    assert err_p > 1e-2
    assert err_b < 10 * 0.7 ** 60 and abs(lb[0]) < 10 * 0.7 ** 60


def test_start_vector_offset_draws_the_next_counters():
    a = O.start_vectors(7, 3, 4, offset=8)
    b = O.start_vectors(7, 3, 8)
    np.testing.assert_array_equal(a, b[:, 4:])


def test_gpu_recipe_generator_equals_numpy_recipe_without_noise():
    """phantoms_torch draws the same parameters as phantoms.make_case; without noise the
    calibration blocks agree to rounding (evaluated here on the CPU device)."""
    torch = pytest.importorskip("torch")
    from paper_2302_13431_gb300.phantoms import make_case
    from paper_2302_13431_gb300.phantoms_torch import make_calib
    for grid, Q, cs in (((32, 40), 4, (12, 10)), ((16, 12, 14), 3, (8, 6, 8))):
        ref = make_case(grid, Q, cs, seed=5, noise=0.0).calib
        got, _ = make_calib(grid, Q, cs, seed=5, noise=0.0, device="cpu")
        got = got.numpy()
        assert np.abs(got - ref).max() <= 1e-6 * np.abs(ref).max()
