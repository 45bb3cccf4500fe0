"""Exact masked Gram (PISCO_FLAG_MASKED_GRAM): the Gram of the calibration matrix restricted to
the rows n with n - Lambda inside the box, against the oracle's explicit C_valid^H C_valid, and
the whole estimate against the oracle run with the masked matrix."""
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

import test_gpu_parity as P  # noqa: E402  (shared case table and gating helpers)


@pytest.mark.parametrize("name", ["2d_small_rect", "2d_ragged", "3d_small", "2d_q33"])
def test_masked_gram_equals_valid_rows_gram(name):
    grid, Q, cs, tau, shape, red, iters, phase = P.CASES[name]
    case = make_case(grid, Q, cs, seed=3, phase=phase)
    D = len(grid)
    tt = tuple([tau] * D) if isinstance(tau, int) else tuple(tau)
    lam = O.kernel_support(tt, shape)
    C = O.calibration_matrix(case.calib, lam, rows="valid")
    A_ref = C.conj().T @ C
    est = PiscoEstimator(grid, cs, Q, tau, kernel_shape=shape, reduction=red, iters=iters, masked_gram=True)
    est(torch.from_numpy(case.calib).cuda())
    n = A_ref.shape[0]
    A = est.debug_buffer(B.PISCO_BUF_GRAM).cpu().numpy().reshape(n, n)
    err = np.abs(A - A_ref).max() / np.abs(A_ref).max()
    assert err <= 1e-11, err
    assert np.array_equal(A, A.conj().T)  # exactly Hermitian by construction
    est.close()


@pytest.mark.parametrize("name", ["2d_small_rect", "2d_256_q32"])
def test_masked_estimate_matches_oracle_with_valid_rows(name):
    grid, Q, cs, tau, shape, red, iters, phase = P.CASES[name]
    case = make_case(grid, Q, cs, seed=0, phase=phase)
    ref = O.estimate(case.calib, grid, tau, shape=shape, reduction=red, iters=iters, seed=0, rows="valid",
                     return_all=True, exact=False)
    est = PiscoEstimator(grid, cs, Q, tau, kernel_shape=shape, reduction=red, iters=iters, masked_gram=True)
    maps, eig = est(torch.from_numpy(case.calib).cuda())
    torch.cuda.synchronize()
    assert est.info()["k"] == ref["U_sig"].shape[1]
    r = dict(case=case, ref=ref, grid=grid, red=red)
    m = P._gated_mask(r).reshape(-1)
    a = maps.cpu().numpy().reshape(Q, -1).T
    b = ref["maps"].reshape(Q, -1).T
    err = np.linalg.norm((P._align(a) - P._align(b))[m]) / np.linalg.norm(b[m])
    assert err <= 1e-4, err
    mr = P._gated_mask(r, reduced=True).reshape(-1)
    assert np.abs(eig.cpu().numpy().reshape(-1) - ref["eig"].reshape(-1))[mr].max() <= 1e-5
    est.close()


def test_masked_gram_at_the_3d_calibration_size():
    """The 24^3 calibration box of the 3D workload (sphere r = 3), Q = 4: the masked Gram equals
    the oracle's explicit C_valid^H C_valid (5832 valid rows)."""
    grid, Q, cs, tau = (48, 48, 48), 4, (24, 24, 24), 3
    case = make_case(grid, Q, cs, seed=5)
    lam = O.kernel_support((tau,) * 3, "ellipsoid")
    C = O.calibration_matrix(case.calib, lam, rows="valid")
    A_ref = C.conj().T @ C
    est = PiscoEstimator(grid, cs, Q, tau, reduction=4, iters=30, masked_gram=True)
    est(torch.from_numpy(case.calib).cuda())
    torch.cuda.synchronize()
    assert est.last_status == B.PISCO_OK
    n = A_ref.shape[0]
    A = est.debug_buffer(B.PISCO_BUF_GRAM).cpu().numpy().reshape(n, n)
    err = np.abs(A - A_ref).max() / np.abs(A_ref).max()
    assert err <= 1e-11, err
    est.close()


def test_masked_gram_rejects_calibration_beyond_one_tile():
    with pytest.raises(B.PiscoError) as ei:  # 25^3 = 15625 samples > 14528
        PiscoEstimator((100, 100, 100), (25, 25, 25), 4, 3, reduction=4, masked_gram=True)
    assert ei.value.status == B.PISCO_ERR_UNSUPPORTED
