"""The nullspace split is certified in FP64 (threshold footnote of Sec. III-B): on thresholds placed
adversarially close to an eigenvalue of C^H C, the estimator either returns the exact split of
LAPACK's FP64 eigenvalues with PISCO_OK, or reports PISCO_ERR_NOT_CONVERGED.  It never reports
PISCO_OK with a wrong signal dimension.

thr is chosen so that thr^2 lambda_1 = lambda_j (1 +- delta) for an eigenvalue lambda_j next to the
workload's natural split; delta = 1e-2 .. 1e-4 must be certified (the FP64 residual bounds of
converged FP32 Ritz vectors are far smaller), smaller delta may end either way."""
import numpy as np
import pytest

from oracle import pisco_oracle as O
from paper_2302_13431_gb300.phantoms import make_case

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_13431_gb300 import _binding as B  # noqa: E402
from paper_2302_13431_gb300.estimator import PiscoEstimator  # noqa: E402

CASES = {
    # name: grid, Q, calib, tau, shape, reduction, extra estimator options
    "2d_small_rect": ((64, 64), 8, (24, 24), 2, "rect", 1, {}),
    "2d_256_q32_tuned": ((256, 256), 32, (32, 32), 3, "ellipsoid", 4,
                         dict(precision="tc_g_eig", tc_splits=1, gemm_splits=2, gemm_tile=64, gram_df=True,
                              tc_interp=True)),
}
_spectra = {}


def _spectrum(name):
    if name not in _spectra:
        grid, Q, cs, tau, shape, red, _ = CASES[name]
        case = make_case(grid, Q, cs, seed=21, phase="poly4")
        D = len(grid)
        lam = O.kernel_support((tau,) * D, shape)
        C = O.calibration_matrix(case.calib, lam, rows="full")
        w = np.linalg.eigvalsh(C.conj().T @ C)[::-1]
        _, U_sig, _ = O.nullspace_svd(C, 0.05)
        _spectra[name] = (case, w, U_sig.shape[1])
    return _spectra[name]


def _run(name, thr, eig_iters=0):
    grid, Q, cs, tau, shape, red, kw = CASES[name]
    case, w, _ = _spectrum(name)
    est = PiscoEstimator(grid, cs, Q, tau, kernel_shape=shape, thr=thr, reduction=red, iters=10,
                         eig_iters=eig_iters, **kw)
    calib = torch.from_numpy(case.calib).cuda()
    maps = torch.empty((Q,) + grid, dtype=torch.complex64, device="cuda")
    st = B.pisco_estimate(est._plan, calib.data_ptr(), maps.data_ptr(), None)
    torch.cuda.synchronize()
    out = (st, est.info()["k"], est.stats())
    est.close()
    return out


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("offset", [-1, 0, 1])
@pytest.mark.parametrize("side", [+1, -1])
@pytest.mark.parametrize("delta", [1e-2, 1e-3, 1e-4, 1e-6, 1e-9])
def test_adversarial_threshold(name, offset, side, delta):
    case, w, k_nat = _spectrum(name)
    j = k_nat + offset                     # eigenvalue index placed at the threshold
    theta = w[j] * (1 + side * delta)      # theta = thr^2 lambda_1
    thr = float(np.sqrt(theta / w[0]))
    k_exp = int((w >= thr * thr * w[0]).sum())
    assert k_exp == (j if side > 0 else j + 1)
    st, k, stats = _run(name, thr)
    if delta >= 1e-4:
        assert st == B.PISCO_OK, (st, stats)
    assert st in (B.PISCO_OK, B.PISCO_ERR_NOT_CONVERGED), st
    if st == B.PISCO_OK:
        assert k == k_exp, (k, k_exp, stats)
        assert stats["cert_margin"] > 0
    print(f"{name} j={j} side={side:+d} delta={delta:.0e}: status {st}, k {k} (LAPACK {k_exp}), "
          f"margin {stats['cert_margin']:.2e}, resid {stats['band_resid']:.2e}, iters {stats['eig_iters']}")


@pytest.mark.parametrize("name", sorted(CASES))
@pytest.mark.parametrize("eig_iters", [1, 2, 3])
def test_too_few_iterations_never_report_a_wrong_split(name, eig_iters):
    """With a fixed (too small) iteration count there is no retry: an unconverged block must show
    as PISCO_ERR_NOT_CONVERGED, never as PISCO_OK with a wrong k."""
    case, w, k_nat = _spectrum(name)
    for offset in (0, 1):
        theta = w[k_nat + offset] * (1 + 1e-3)
        thr = float(np.sqrt(theta / w[0]))
        k_exp = int((w >= thr * thr * w[0]).sum())
        st, k, stats = _run(name, thr, eig_iters=eig_iters)
        assert st in (B.PISCO_OK, B.PISCO_ERR_NOT_CONVERGED), st
        if st == B.PISCO_OK:
            assert k == k_exp, (k, k_exp, stats)
