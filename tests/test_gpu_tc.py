"""Tensor-core complex GEMM (tcgen05, split TF32) through the C ABI against an FP64 product.

Error model: a 3-pass product (head*head + head*tail + tail*head, TF32 heads and tails) has a
per-product relative error of about 2^-21 plus FP32 accumulation; a 1-pass product about
2^-11.  The bound is per entry, relative to |A| |op(B)| (the product of the magnitudes), so it
is independent of cancellation in the entry itself.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_13431_gb300 import _binding as B  # noqa: E402

TOL = {3: 2e-5, 1: 2e-3}


def _rand(rng, *shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def _run(nterms, A, Bm, opB, alpha=1.0, beta=0.0, C0=None, pipelined=1):
    """The TMA-fed tensor-core GEMM (pisco_tc_cgemm_pipelined) with `pipelined` K splits."""
    M, K = A.shape
    N = Bm.shape[1] if opB == 0 else Bm.shape[0]
    dA = torch.from_numpy(A).cuda()
    dB = torch.from_numpy(Bm).cuda()
    dC = torch.from_numpy(C0.copy()).cuda() if C0 is not None else torch.zeros((M, N), dtype=torch.complex64,
                                                                                 device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    nb = B.pisco_tc_cgemm_pipelined_workspace(nterms, M, N, K, pipelined)
    ws = torch.empty(max(nb, 16), dtype=torch.uint8, device="cuda")
    st = B.pisco_tc_cgemm_pipelined(nterms, M, N, K, alpha, dA.data_ptr(), K, dB.data_ptr(), Bm.shape[1], opB,
                                    beta, dC.data_ptr(), N, pipelined, ws.data_ptr(), nb, status.data_ptr(),
                                    stream)
    assert st == B.PISCO_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return dC.cpu().numpy()


def _check(nterms, A, Bm, opB, alpha=1.0, beta=0.0, C0=None, pipelined=1):
    A64 = A.astype(np.complex128)
    opb = Bm.astype(np.complex128) if opB == 0 else Bm.astype(np.complex128).conj().T
    ref = alpha * (A64 @ opb)
    mag = np.abs(alpha) * (np.abs(A64) @ np.abs(opb))
    if C0 is not None and beta != 0:
        ref = ref + beta * C0.astype(np.complex128)
        mag = mag + np.abs(beta) * np.abs(C0)
    out = _run(nterms, A, Bm, opB, alpha, beta, C0, pipelined)
    err = np.abs(out - ref) / (mag + 1e-30)
    print(f"tc_cgemm nterms={nterms} A={A.shape} opB={opB} pipelined={pipelined}: "
          f"max error / (|A||B|) = {err.max():.3e}")
    assert err.max() <= TOL[nterms], (nterms, A.shape, opB, err.max())
    return err.max()


@pytest.mark.parametrize("nterms", [3, 1])
@pytest.mark.parametrize("M,N,K", [(128, 32, 16), (200, 50, 37), (928, 64, 928), (300, 1024, 105),
                                   (129, 33, 1), (1, 1, 17)])
def test_tc_gemm_opB_N(nterms, M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    _check(nterms, _rand(rng, M, K), _rand(rng, K, N), 0)


@pytest.mark.parametrize("nterms", [3, 1])
@pytest.mark.parametrize("n,k", [(928, 64), (200, 22), (65, 9)])
def test_tc_gemm_opB_C_hermitian_product(nterms, n, k):
    # P = U diag(w) U^H without the weights: op(B) = conj(U^T)
    rng = np.random.default_rng(n + k)
    U = _rand(rng, n, k)
    _check(nterms, U, U, 1)


def test_tc_gemm_alpha_beta_and_empty_K():
    rng = np.random.default_rng(5)
    A, Bm, C0 = _rand(rng, 150, 40), _rand(rng, 40, 70), _rand(rng, 150, 70)
    _check(3, A, Bm, 0, alpha=0.5 - 2j, beta=-1 + 0.25j, C0=C0)
    # K = 0: C = beta * C
    out = _run(3, np.zeros((150, 0), np.complex64), np.zeros((0, 70), np.complex64), 0, 1.0, 2.0, C0)
    np.testing.assert_allclose(out, 2.0 * C0, rtol=1e-6)


def test_tc_gemm_rejects_bad_arguments():
    d = torch.zeros(64, dtype=torch.complex64, device="cuda")
    p = d.data_ptr()
    ws = torch.empty(1 << 16, dtype=torch.uint8, device="cuda")
    w, nb = ws.data_ptr(), ws.numel()
    assert B.pisco_tc_cgemm_pipelined(2, 4, 4, 4, 1, p, 4, p, 4, 0, 0, p, 4, 1, w, nb) == B.PISCO_ERR_ARG
    assert B.pisco_tc_cgemm_pipelined(3, 4, 4, 4, 1, p, 3, p, 4, 0, 0, p, 4, 1, w, nb) == B.PISCO_ERR_ARG  # lda < K
    assert B.pisco_tc_cgemm_pipelined(3, 4, 4, 4, 1, p + 4, 4, p, 4, 0, 0, p, 4, 1, w, nb) == B.PISCO_ERR_ARG
    assert B.pisco_tc_cgemm_pipelined(3, 4, 4, 4, 1, p, 4, p, 4, 0, 0, p, 4, 1, w, 16) == B.PISCO_ERR_ARG  # small ws
    assert B.pisco_tc_cgemm_pipelined(3, 0, 4, 4, 1, 0, 4, 0, 4, 0, 0, 0, 4, 1, w, nb) == B.PISCO_OK  # empty


@pytest.mark.parametrize("splits", [1, 4])
@pytest.mark.parametrize("nterms", [3, 1])
@pytest.mark.parametrize("M,N,K", [(128, 32, 16), (200, 50, 37), (928, 64, 928), (4096, 1024, 105),
                                   (129, 33, 1), (1, 1, 17)])
def test_pipelined_gemm_opB_N(nterms, M, N, K, splits):
    rng = np.random.default_rng(M * 7 + N * 3 + K + 1)
    _check(nterms, _rand(rng, M, K), _rand(rng, K, N), 0, pipelined=splits)


@pytest.mark.parametrize("splits", [1, 3])
@pytest.mark.parametrize("n,k", [(928, 64), (200, 22), (65, 9)])
def test_pipelined_gemm_opB_C(n, k, splits):
    rng = np.random.default_rng(n + k + 2)
    U = _rand(rng, n, k)
    _check(3, U, U, 1, pipelined=splits)


def test_pipelined_gemm_alpha_beta_split_and_determinism():
    rng = np.random.default_rng(6)
    A, Bm, C0 = _rand(rng, 300, 200), _rand(rng, 200, 70), _rand(rng, 300, 70)
    _check(3, A, Bm, 0, alpha=0.5 - 2j, beta=-1 + 0.25j, C0=C0, pipelined=4)
    a = _run(3, A, Bm, 0, pipelined=4)
    b = _run(3, A, Bm, 0, pipelined=4)
    np.testing.assert_array_equal(a, b)
