"""The allocation-free lag-table entry point (pisco_gram_lags_noalloc) against the lag table
that pisco_estimate computes, through the C ABI, on two calls in a row.

This file is collected last on purpose: if it fails, a run that stops at the first failure
has already run every other test.  It passes alone in a fresh process as well.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_13431_gb300 import _binding as B  # noqa: E402
from paper_2302_13431_gb300.estimator import PiscoEstimator  # noqa: E402
from paper_2302_13431_gb300.phantoms import make_case  # noqa: E402

CASES = [
    # grid, Q, calib, tau, shape
    ((256, 256), 32, (32, 32), 3, "ellipsoid"),
    ((40, 48), 5, (18, 20), (2, 3), "ellipsoid"),
    ((16, 24, 20), 4, (10, 12, 10), 2, "ellipsoid"),
]


@pytest.mark.parametrize("case_idx", range(len(CASES)))
def test_noalloc_lags_match_estimate_lags_twice(case_idx):
    grid, Q, cs, tau, shape = CASES[case_idx]
    case = make_case(grid, Q, cs, seed=21 + case_idx)
    calib = torch.from_numpy(case.calib).cuda()
    est = PiscoEstimator(grid, cs, Q, tau, kernel_shape=shape, reduction=1, iters=2)
    est(calib)
    torch.cuda.synchronize()
    ref = est.debug_buffer(B.PISCO_BUF_LAGS).cpu().numpy()
    est.close()
    params = B.make_params(grid, cs, Q, tau, shape, 0.05, 1, 2)
    lags = torch.full((ref.size,), float("nan"), dtype=torch.complex128, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        lags.fill_(complex(float("nan"), float("nan")))
        st = B.pisco_gram_lags_noalloc(params, calib.data_ptr(), lags.data_ptr(), stream)
        assert st == B.PISCO_OK, B.pisco_status_string(st)
        torch.cuda.synchronize()
        got = lags.cpu().numpy()
        assert np.all(np.isfinite(got))
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= 1e-12, (call, err)


def test_noalloc_rejects_requests_beyond_its_scratch():
    grid, Q, cs, tau = (128, 128, 96), 32, (24, 24, 24), 3
    params = B.make_params(grid, cs, Q, tau, "ellipsoid", 0.05, 4, 2)
    dummy = torch.zeros(16, dtype=torch.complex128, device="cuda")
    st = B.pisco_gram_lags_noalloc(params, dummy.data_ptr(), dummy.data_ptr(), 0)
    assert st == B.PISCO_ERR_TOO_LARGE
