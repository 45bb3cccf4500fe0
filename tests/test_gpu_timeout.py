"""The bounded device waits of the tensor-core products end in a status, not a hang.

With the test hook on, every tensor-core product issues no loads and waits about 10 ms at most:
the waits expire with nothing in flight, the kernel frees its tensor memory and sets bit 16 of
the status word, and pisco_estimate returns PISCO_ERR_TIMEOUT.  With the hook off again the
same plan (and the same process) gives bitwise the result of a fresh plan."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_13431_gb300 import _binding as B  # noqa: E402
from paper_2302_13431_gb300.estimator import PiscoEstimator  # noqa: E402
from paper_2302_13431_gb300.phantoms import make_case  # noqa: E402


def _gemm_status(M, N, K):
    rng = np.random.default_rng(1)
    A = torch.from_numpy((rng.standard_normal((M, K)) + 1j * rng.standard_normal((M, K))).astype(np.complex64)).cuda()
    Bm = torch.from_numpy((rng.standard_normal((K, N)) + 1j * rng.standard_normal((K, N))).astype(np.complex64)).cuda()
    C = torch.zeros((M, N), dtype=torch.complex64, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    nb = B.pisco_tc_cgemm_pipelined_workspace(3, M, N, K, 1)
    ws = torch.empty(nb, dtype=torch.uint8, device="cuda")
    st = B.pisco_tc_cgemm_pipelined(3, M, N, K, 1.0, A.data_ptr(), K, Bm.data_ptr(), N, 0, 0.0, C.data_ptr(), N, 1,
                                    ws.data_ptr(), nb, status.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st, int(status.item()), C, (A.cpu().numpy().astype(np.complex128) @ Bm.cpu().numpy())


def test_expired_waits_set_the_status_bit_and_leave_the_context_usable():
    B.pisco_test_stall_tensor_loads(True)
    try:
        st, flags, _, _ = _gemm_status(256, 64, 96)
    finally:
        B.pisco_test_stall_tensor_loads(False)
    assert st == B.PISCO_OK and (flags & 16)
    st, flags, C, ref = _gemm_status(256, 64, 96)
    assert st == B.PISCO_OK and flags == 0
    assert np.abs(C.cpu().numpy() - ref).max() <= 1e-4 * np.abs(ref).max()


def test_estimate_reports_timeout_then_recovers_bitwise():
    grid, Q, cs = (64, 64), 8, (24, 24)
    case = make_case(grid, Q, cs, seed=77)
    calib = torch.from_numpy(case.calib).cuda()
    kw = dict(reduction=2, iters=20, precision="tc_g_eig", gram_df=True, tc_interp=True)
    est = PiscoEstimator(grid, cs, Q, 3, **kw)
    maps = torch.empty((Q,) + grid, dtype=torch.complex64, device="cuda")
    eig = torch.empty((32, 32), dtype=torch.float32, device="cuda")
    B.pisco_test_stall_tensor_loads(True)
    try:
        st = B.pisco_estimate(est._plan, calib.data_ptr(), maps.data_ptr(), eig.data_ptr())
    finally:
        B.pisco_test_stall_tensor_loads(False)
    torch.cuda.synchronize()
    assert st == B.PISCO_ERR_TIMEOUT
    st = B.pisco_estimate(est._plan, calib.data_ptr(), maps.data_ptr(), eig.data_ptr())
    torch.cuda.synchronize()
    assert st == B.PISCO_OK
    fresh = PiscoEstimator(grid, cs, Q, 3, **kw)
    m2, e2 = fresh(calib)
    torch.cuda.synchronize()
    assert torch.equal(maps, m2) and torch.equal(eig, e2)
    est.close()
    fresh.close()
