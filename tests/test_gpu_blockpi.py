"""Block power iteration (PISCO_FLAG_BLOCK_PI) and the support mask.

* Stage parity: on the GPU's own G(x) (whose parity is tested elsewhere), the CUDA block
  iteration equals the FP64 oracle's block iteration from the same two counter-based starts,
  after the same phase step.
* Where the two smallest eigenvalues of G(x) are close, the block iteration ends nearer to the
  exact null vector than the single-vector iteration with the same count.
* pisco_support_mask is eig < threshold.
"""
import numpy as np
import pytest
from scipy import ndimage

from oracle import pisco_oracle as O
from paper_2302_13431_gb300.phantoms import make_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_13431_gb300 import _binding as B  # noqa: E402
from paper_2302_13431_gb300.estimator import PiscoEstimator  # noqa: E402

import test_gpu_parity as P  # noqa: E402


def _run(name, block, seed=0):
    grid, Q, cs, tau, shape, red, iters, phase = P.CASES[name]
    case = make_case(grid, Q, cs, seed=seed, phase=phase)
    est = PiscoEstimator(grid, cs, Q, tau, kernel_shape=shape, reduction=red, iters=iters, block_pi=block)
    maps, eig = est(torch.from_numpy(case.calib).cuda())
    torch.cuda.synchronize()
    G = est.debug_buffer(B.PISCO_BUF_G).cpu().numpy().reshape(-1, Q, Q).astype(np.complex128)
    Y = est.debug_buffer(B.PISCO_BUF_Y).cpu().numpy().reshape(Q, -1).T.astype(np.complex128)
    V = est.debug_buffer(B.PISCO_BUF_V).cpu().numpy().reshape(Q, -1).T
    out = dict(case=case, est=est, G=G, Y=Y, V=V, eig=eig.cpu().numpy().reshape(-1), Q=Q, iters=iters,
               grid=grid, red=red, tau=tau, shape=shape)
    return out


def _inner(r):
    inner = ndimage.binary_erosion(np.abs(r["case"].rho) > 0, iterations=2)
    sl = tuple(slice(None, None, r["red"]) for _ in r["grid"])
    return inner[sl].reshape(-1)


@pytest.mark.parametrize("name", ["2d_small_rect", "3d_small", "2d_256_q32"])
def test_block_iteration_matches_oracle(name):
    r = _run(name, True)
    Q, G = r["Q"], r["G"]
    D = len(r["grid"])
    tt = tuple([r["tau"]] * D) if isinstance(r["tau"], int) else tuple(r["tau"])
    L = O.kernel_support(tt, r["shape"]).shape[0]
    npix = G.shape[0]
    V0 = np.stack([O.start_vectors(0, npix, Q), O.start_vectors(0, npix, Q, offset=2 * Q)], axis=2)
    v, lam = O.block_power_iteration(G, V0, r["iters"], L)
    v = O.phase_align(v, r["Y"])
    w = np.linalg.eigvalsh(G) / L
    sel = _inner(r) & ((w[:, 1] - w[:, 0]) > 1e-3)
    assert sel.sum() >= 5
    al = lambda a: a * np.exp(-1j * np.angle(a[:, :1]))  # noqa: E731
    err = np.linalg.norm((al(r["V"]) - al(v))[sel]) / np.linalg.norm(v[sel])
    assert err <= 1e-4, err
    assert np.abs(r["eig"] - lam)[sel].max() <= 1e-5
    r["est"].close()


def test_block_iteration_helps_small_gap_pixels():
    name = "2d_256_q32"
    rb, rp = _run(name, True), _run(name, False)
    G, Q = rb["G"], rb["Q"]
    w, U = np.linalg.eigh(G)
    L = O.kernel_support((3, 3), "ellipsoid").shape[0]
    gap = (w[:, 1] - w[:, 0]) / L
    small = gap < np.percentile(gap, 10)
    vstar = U[:, :, 0]
    eb = 1 - np.abs(np.sum(np.conj(rb["V"]) * vstar, axis=1))
    ep = 1 - np.abs(np.sum(np.conj(rp["V"]) * vstar, axis=1))
    print(f"small-gap pixels {small.sum()}: median 1-|<v,v*>| block {np.median(eb[small]):.2e}, "
          f"single {np.median(ep[small]):.2e}")
    assert np.median(eb[small]) <= np.median(ep[small])
    rb["est"].close()
    rp["est"].close()


def test_support_mask_is_eigenvalue_threshold():
    r = _run("2d_small_rect", False)
    eig = torch.from_numpy(r["eig"]).cuda()
    mask = r["est"].support_mask(eig, 0.05)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(mask.cpu().numpy(), (r["eig"] < 0.05).astype(np.uint8))
    r["est"].close()
