"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle, stage by stage and
end to end, on seeded synthetic data.

Tolerances (derived from the arithmetic of each stage):
  * Gram (FP64 on both sides): max |A_gpu - A_oracle| <= 1e-11 * max|A|.
  * signal dimension k: exact (integer decision taken on FP64 Rayleigh quotients).
  * signal projector U U^H (FP32 subspace iteration): max abs entry error <= 2e-5.
  * G(x) (FP32 assembly): max |G_gpu - G_oracle| <= 2e-5 * |Lambda|.
  * maps: relative L2 error after per-pixel channel-1 phase alignment <= 1e-4 inside the
    phantom support eroded by 2 pixels, at pixels whose eigen-gap (lambda_2 - lambda_1)/|Lambda|
    exceeds 1e-3; eigenvalue map |lambda_gpu - lambda_oracle| <= 1e-5 on the [0,1] scale.
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

CASES = {
    # name: grid, Q, calib, tau, shape, reduction, iters, phase
    "2d_small_rect": ((64, 64), 8, (24, 24), 2, "rect", 1, 30, "linear"),
    "2d_ragged": ((40, 48), 5, (18, 20), (2, 3), "ellipsoid", 2, 30, "poly4"),
    "2d_q33": ((48, 48), 33, (20, 20), 2, "ellipsoid", 2, 20, "poly4"),
    "3d_small": ((16, 24, 20), 4, (10, 12, 10), 2, "ellipsoid", 2, 30, "poly4"),
    "2d_256_q32": ((256, 256), 32, (32, 32), 3, "ellipsoid", 4, 30, "poly4"),
    # fused per-pixel normalisation over 16 / 8 coil rows; ragged row and column tiles
    "2d_q16": ((64, 80), 16, (20, 20), 2, "ellipsoid", 2, 30, "poly4"),
    "2d_q8": ((72, 96), 8, (24, 24), 2, "ellipsoid", 4, 30, "poly4"),
}
_cache = {}


_refs = {}


def _oracle(name, seed):
    if (name, seed) not in _refs:
        grid, Q, cs, tau, shape, red, iters, phase = CASES[name]
        case = make_case(grid, Q, cs, seed=seed, phase=phase)
        ref = O.estimate(case.calib, grid, tau, shape=shape, reduction=red, iters=iters, seed=seed,
                         return_all=True, exact=False)
        _refs[(name, seed)] = (case, ref)
    return _refs[(name, seed)]


def _run(name, seed=0, precision="fp32"):
    key = (name, seed, precision)
    if key in _cache:
        return _cache[key]
    grid, Q, cs, tau, shape, red, iters, phase = CASES[name]
    case, ref = _oracle(name, seed)
    est = PiscoEstimator(grid, cs, Q, tau, kernel_shape=shape, reduction=red, iters=iters, seed=seed,
                         precision=precision)
    maps, eig = est(torch.from_numpy(case.calib).cuda())
    torch.cuda.synchronize()
    out = dict(case=case, ref=ref, est=est, maps=maps.cpu().numpy(), eig=eig.cpu().numpy(),
               grid=grid, Q=Q, red=red, tau=tau, shape=shape, status=est.last_status)
    out["A"] = est.debug_buffer(B.PISCO_BUF_GRAM).cpu().numpy()
    out["U"] = est.debug_buffer(B.PISCO_BUF_SIGNAL).cpu().numpy()
    out["w"] = est.debug_buffer(B.PISCO_BUF_WEIGHTS).cpu().numpy()
    out["ritz"] = est.debug_buffer(B.PISCO_BUF_RITZ).cpu().numpy()
    out["G"] = est.debug_buffer(B.PISCO_BUF_G).cpu().numpy()
    out["V"] = est.debug_buffer(B.PISCO_BUF_V).cpu().numpy()
    out["Y"] = est.debug_buffer(B.PISCO_BUF_Y).cpu().numpy()
    out["info"] = est.info()
    _cache[key] = out
    return out


def _align(v):
    """Per-pixel phase alignment to channel 1 (v: [npix, Q])."""
    ph = np.exp(-1j * np.angle(v[:, :1]))
    return v * ph


def _gated_mask(r, reduced=False):
    case, ref = r["case"], r["ref"]
    supp = np.abs(case.rho) > 0
    inner = ndimage.binary_erosion(supp, iterations=2)
    red = r["red"]
    if reduced:
        sl = tuple(slice(None, None, red) for _ in r["grid"])
        inner = inner[sl]
    # gap from LAPACK eigenvalues of the oracle's G (library route, reduced grid)
    w = np.linalg.eigvalsh(ref["G"]) / ref["lam"].shape[0]
    gap = (w[:, 1] - w[:, 0]).reshape(tuple(g // red for g in r["grid"]))
    if reduced:
        return inner & (gap > 1e-3)
    # full grid: a pixel counts when its nearest reduced pixel is gapped
    up = gap
    for ax in range(gap.ndim):
        up = np.repeat(up, red, axis=ax)
    return inner & (up > 1e-3)


@pytest.mark.parametrize("name", ["2d_small_rect", "2d_ragged", "3d_small", "2d_q33"])
def test_gram_matches_explicit_CtC(name):
    r = _run(name)
    C = r["ref"]["C"]
    A_ref = C.conj().T @ C
    n = A_ref.shape[0]
    A = r["A"].reshape(n, n)
    err = np.abs(A - A_ref).max() / np.abs(A_ref).max()
    assert err <= 1e-11, err


@pytest.mark.parametrize("name", ["2d_small_rect", "2d_ragged", "3d_small", "2d_q33", "2d_256_q32"])
def test_nullspace_split_and_projector(name):
    r = _run(name)
    ref = r["ref"]
    k_ref = ref["U_sig"].shape[1]
    assert r["info"]["k"] == k_ref
    assert r["info"]["R"] == ref["V_null"].shape[1]
    n = ref["U_sig"].shape[0]
    m = r["w"].shape[0]
    U = r["U"].reshape(n, m)[:, r["w"] > 0].astype(np.complex128)
    P = U @ U.conj().T
    P_ref = ref["U_sig"] @ ref["U_sig"].conj().T
    err = np.abs(P - P_ref).max()
    assert err <= 2e-5, err
    # FP64 Rayleigh quotients of the decided Ritz values against LAPACK
    lam = np.sort(ref["sigma"] ** 2)[::-1]
    ritz = r["ritz"]
    assert abs(ritz[0] - lam[0]) <= 1e-9 * lam[0]


@pytest.mark.parametrize("name", ["2d_small_rect", "2d_ragged", "3d_small", "2d_q33", "2d_256_q32"])
def test_G_field(name):
    r = _run(name)
    ref = r["ref"]
    Q = r["Q"]
    L = ref["lam"].shape[0]
    npix = ref["G"].shape[0]
    G = r["G"].reshape(npix, Q, Q)
    err = np.abs(G - ref["G"]).max() / L
    assert err <= 2e-5, err


@pytest.mark.parametrize("name", ["2d_small_rect", "2d_ragged", "3d_small", "2d_q33", "2d_256_q32"])
def test_lowres_images(name):
    r = _run(name)
    Q = r["Q"]
    Y = r["Y"].reshape(Q, -1).T
    ref = r["ref"]["y"]
    err = np.abs(Y - ref).max() / np.abs(ref).max()
    assert err <= 1e-5, err


@pytest.mark.parametrize("name", ["2d_small_rect", "2d_ragged", "3d_small", "2d_q33", "2d_256_q32"])
def test_power_iteration_phase_and_eig(name):
    r = _run(name)
    Q = r["Q"]
    m = _gated_mask(r, reduced=True).reshape(-1)
    v = r["V"].reshape(Q, -1).T
    vr = r["ref"]["v_aligned"]
    err = np.linalg.norm((_align(v) - _align(vr))[m]) / np.linalg.norm(vr[m])
    assert err <= 1e-4, err
    eerr = np.abs(r["eig"].reshape(-1) - r["ref"]["eig"].reshape(-1))[m].max()
    assert eerr <= 1e-5, eerr


@pytest.mark.parametrize("name", ["2d_small_rect", "2d_ragged", "3d_small", "2d_q33", "2d_256_q32"])
def test_end_to_end_maps(name):
    r = _run(name)
    Q = r["Q"]
    a = r["maps"].reshape(Q, -1).T
    b = r["ref"]["maps"].reshape(Q, -1).T
    m = _gated_mask(r).reshape(-1)
    err = np.linalg.norm((_align(a) - _align(b))[m]) / np.linalg.norm(b[m])
    assert err <= 1e-4, err
    nrm = np.linalg.norm(a, axis=1)
    assert np.all((np.abs(nrm - 1) < 1e-5) | (nrm == 0))


def test_host_entry_point_matches_device_entry_point():
    grid, Q, cs, tau, shape, red, iters, phase = CASES["2d_ragged"]
    case = make_case(grid, Q, cs, seed=4, phase=phase)
    est = PiscoEstimator(grid, cs, Q, tau, kernel_shape=shape, reduction=red, iters=iters, host_io=True)
    maps_d, eig_d = est(torch.from_numpy(case.calib).cuda())
    maps_h = np.empty((Q,) + grid, np.complex64)
    eig_h = np.empty(tuple(g // red for g in grid), np.float32)
    est.estimate_host(case.calib, maps_h, eig_h)
    np.testing.assert_array_equal(maps_h, maps_d.cpu().numpy())
    np.testing.assert_array_equal(eig_h, eig_d.cpu().numpy())
    est.close()


def test_repeated_calls_are_deterministic():
    r = _run("2d_ragged")
    est = r["est"]
    calib = torch.from_numpy(r["case"].calib).cuda()
    m1, e1 = est(calib)
    m2, e2 = est(calib)
    torch.cuda.synchronize()
    assert torch.equal(m1, m2) and torch.equal(e1, e2)


def test_zero_calibration_reports_rank_failure():
    grid, Q, cs, tau = (32, 32), 4, (12, 12), 2
    est = PiscoEstimator(grid, cs, Q, tau, kernel_shape="rect")
    calib = torch.zeros((Q,) + cs, dtype=torch.complex64, device="cuda")
    maps = torch.empty((Q,) + grid, dtype=torch.complex64, device="cuda")
    st = est.estimate_into(calib, maps, None)
    assert st == B.PISCO_ERR_RANK
    assert bool(torch.isfinite(torch.view_as_real(maps)).all())
    est.close()


def test_invalid_arguments_are_rejected_without_launch():
    grid, Q, cs = (32, 32), 4, (12, 12)
    est = PiscoEstimator(grid, cs, Q, 2, kernel_shape="rect")
    calib = torch.zeros((Q,) + cs, dtype=torch.complex64, device="cuda")
    assert B.pisco_estimate(est._plan, calib.data_ptr(), 0, None) == B.PISCO_ERR_ARG
    assert B.pisco_estimate(est._plan, calib.data_ptr() + 4, calib.data_ptr(), None) == B.PISCO_ERR_ARG
    est.close()


def test_graph_replay_reads_new_calibration_data():
    """Same buffers on every call: the first call runs eagerly, the second captures a CUDA graph,
    the third replays it.  The replay must pick up the new contents of the calibration buffer."""
    grid, Q, cs, tau, shape, red, iters, phase = CASES["2d_ragged"]
    a = make_case(grid, Q, cs, seed=11, phase=phase).calib
    b = make_case(grid, Q, cs, seed=12, phase=phase).calib
    est = PiscoEstimator(grid, cs, Q, tau, kernel_shape=shape, reduction=red, iters=iters)
    calib = torch.from_numpy(a).cuda()
    maps = torch.empty((Q,) + grid, dtype=torch.complex64, device="cuda")
    eig = torch.empty(tuple(g // red for g in grid), dtype=torch.float32, device="cuda")
    est.estimate_into(calib, maps, eig)
    first = maps.clone()
    est.estimate_into(calib, maps, eig)
    assert torch.equal(first, maps)
    calib.copy_(torch.from_numpy(b))
    est.estimate_into(calib, maps, eig)
    fresh = PiscoEstimator(grid, cs, Q, tau, kernel_shape=shape, reduction=red, iters=iters)
    maps_b, eig_b = fresh(torch.from_numpy(b).cuda())
    torch.cuda.synchronize()
    assert torch.equal(maps, maps_b) and torch.equal(eig, eig_b)
    est.close()
    fresh.close()


# ---- split-precision tensor-core routes (G(x) assembly, eigensolver block products) ----------
TC_CASES = ["2d_small_rect", "2d_ragged", "2d_q33", "3d_small", "2d_256_q32"]


def _errors(r):
    """Per-output errors against the FP64 oracle: k, projector, G, PI vectors, eig, maps."""
    ref, Q = r["ref"], r["Q"]
    n = ref["U_sig"].shape[0]
    m = r["w"].shape[0]
    U = r["U"].reshape(n, m)[:, r["w"] > 0].astype(np.complex128)
    P_err = np.abs(U @ U.conj().T - ref["U_sig"] @ ref["U_sig"].conj().T).max()
    L = ref["lam"].shape[0]
    G_err = np.abs(r["G"].reshape(-1, Q, Q) - ref["G"]).max() / L
    mr = _gated_mask(r, reduced=True).reshape(-1)
    v = r["V"].reshape(Q, -1).T
    vr = ref["v_aligned"]
    v_err = np.linalg.norm((_align(v) - _align(vr))[mr]) / np.linalg.norm(vr[mr])
    e_err = np.abs(r["eig"].reshape(-1) - ref["eig"].reshape(-1))[mr].max()
    mf = _gated_mask(r).reshape(-1)
    a = r["maps"].reshape(Q, -1).T
    b = ref["maps"].reshape(Q, -1).T
    map_err = np.linalg.norm((_align(a) - _align(b))[mf]) / np.linalg.norm(b[mf])
    return dict(k_ok=r["info"]["k"] == ref["U_sig"].shape[1], projector=P_err, G=G_err, pi=v_err,
                eig=e_err, maps=map_err)


@pytest.mark.parametrize("precision", ["tc_g", "tc_g_eig", "tc_all"])
@pytest.mark.parametrize("name", TC_CASES)
def test_split_tf32_routes_meet_fp32_tolerances(name, precision):
    r = _run(name, precision=precision)
    e = _errors(r)
    print(f"{name} {precision}: " + " ".join(f"{k}={v:.2e}" if not isinstance(v, bool) else f"{k}={v}"
                                             for k, v in e.items()))
    assert e["k_ok"]
    assert e["projector"] <= 2e-5
    assert e["G"] <= 2e-5
    assert e["pi"] <= 1e-4 and e["eig"] <= 1e-5
    assert e["maps"] <= 1e-4


@pytest.mark.parametrize("name", ["2d_q33", "2d_256_q32"])
def test_single_pass_tf32_error_is_reported(name):
    """One TF32 pass per product: about 11 significant bits in G.  Its error is reported against
    the oracle; it is bounded here by what the 2^-11 operand rounding allows, not by the FP32 gate."""
    r = _run(name, precision="tc_g_1pass")
    e = _errors(r)
    print(f"{name} tc_g_1pass: " + " ".join(f"{k}={v:.2e}" if not isinstance(v, bool) else f"{k}={v}"
                                            for k, v in e.items()))
    assert e["k_ok"]
    assert e["G"] <= 2e-3
    assert np.isfinite(r["maps"]).all()


# ---- the Gram's FFT route in double-float arithmetic (PISCO_FLAG_GRAM_DF) ----------------------
@pytest.mark.parametrize("name", ["2d_small_rect", "2d_ragged", "3d_small", "2d_q33", "2d_256_q32"])
def test_double_float_gram_matches_explicit_CtC_and_maps(name):
    grid, Q, cs, tau, shape, red, iters, phase = CASES[name]
    case, ref = _oracle(name, 0)
    est = PiscoEstimator(grid, cs, Q, tau, kernel_shape=shape, reduction=red, iters=iters, gram_df=True)
    maps, eig = est(torch.from_numpy(case.calib).cuda())
    torch.cuda.synchronize()
    C = ref["C"]
    A_ref = C.conj().T @ C
    n = A_ref.shape[0]
    A = est.debug_buffer(B.PISCO_BUF_GRAM).cpu().numpy().reshape(n, n)
    err = np.abs(A - A_ref).max() / np.abs(A_ref).max()
    print(f"{name}: double-float Gram max error / max|A| = {err:.2e}")
    assert err <= 1e-11, err
    assert est.info()["k"] == ref["U_sig"].shape[1]
    r = dict(case=case, ref=ref, grid=grid, red=red)
    m = _gated_mask(r).reshape(-1)
    a = maps.cpu().numpy().reshape(Q, -1).T
    b = ref["maps"].reshape(Q, -1).T
    assert np.linalg.norm((_align(a) - _align(b))[m]) / np.linalg.norm(b[m]) <= 1e-4
    est.close()


# ---- the last interpolation pass on the tensor cores (PISCO_FLAG_TC_INTERP) --------------------
@pytest.mark.parametrize("name", ["2d_small_rect", "2d_ragged", "3d_small", "2d_q33", "2d_256_q32", "2d_q16", "2d_q8"])
def test_tensor_core_interpolation_matches_oracle_and_fp32_route(name):
    """maps_q = M T_q as one batched split-TF32 GEMM, then the per-pixel normalisation: the same
    map gate as the FP32 route, and within 1e-5 of the FP32 route's maps on the gated pixels.
    (2d_small_rect has no grid reduction, so the flag leaves its path unchanged.)"""
    grid, Q, cs, tau, shape, red, iters, phase = CASES[name]
    case, ref = _oracle(name, 0)
    est = PiscoEstimator(grid, cs, Q, tau, kernel_shape=shape, reduction=red, iters=iters, tc_interp=True)
    maps, eig = est(torch.from_numpy(case.calib).cuda())
    torch.cuda.synchronize()
    r0 = _run(name)
    r = dict(case=case, ref=ref, grid=grid, red=red)
    m = _gated_mask(r).reshape(-1)
    a = maps.cpu().numpy().reshape(Q, -1).T
    b = ref["maps"].reshape(Q, -1).T
    a0 = r0["maps"].reshape(Q, -1).T
    err = np.linalg.norm((_align(a) - _align(b))[m]) / np.linalg.norm(b[m])
    d32 = np.linalg.norm((a - a0)[m]) / np.linalg.norm(a0[m])
    print(f"{name}: tc interp maps error vs oracle {err:.2e}, vs FP32 route {d32:.2e}")
    assert err <= 1e-4, err
    assert d32 <= 1e-5, d32
    nrm = np.linalg.norm(a, axis=1)
    assert np.all((np.abs(nrm - 1) < 1e-5) | (nrm == 0))
    np.testing.assert_array_equal(eig.cpu().numpy(), r0["eig"])
    est.close()


# ---- 2D G(x): separable DFT passes (default of the tensor-core G route) vs the dense lag GEMM ---
@pytest.mark.parametrize("name", ["2d_small_rect", "2d_ragged", "2d_q33", "2d_256_q32"])
def test_separable_and_dense_G_routes_agree(name):
    """Both evaluations of sum_d K_pq[d] exp(i 2 pi d x) meet the FP32 G gate against the oracle
    and agree with each other within it; the maps of the separable route meet the map gate."""
    grid, Q, cs, tau, shape, red, iters, phase = CASES[name]
    case, ref = _oracle(name, 0)
    out = {}
    for dense in (False, True):
        est = PiscoEstimator(grid, cs, Q, tau, kernel_shape=shape, reduction=red, iters=iters, precision="tc_g",
                             g_dense=dense)
        maps, _ = est(torch.from_numpy(case.calib).cuda())
        torch.cuda.synchronize()
        out[dense] = (est.debug_buffer(B.PISCO_BUF_G).cpu().numpy().reshape(-1, Q, Q), maps.cpu().numpy())
        est.close()
    L = ref["lam"].shape[0]
    e_sep = np.abs(out[False][0] - ref["G"]).max() / L
    e_den = np.abs(out[True][0] - ref["G"]).max() / L
    e_rt = np.abs(out[False][0] - out[True][0]).max() / L
    print(f"{name}: G error / |Lambda|: separable {e_sep:.2e}, dense {e_den:.2e}, between {e_rt:.2e}")
    assert e_sep <= 2e-5 and e_den <= 2e-5 and e_rt <= 2e-5
    r = dict(case=case, ref=ref, grid=grid, red=red)
    m = _gated_mask(r).reshape(-1)
    a = out[False][1].reshape(Q, -1).T
    b = ref["maps"].reshape(Q, -1).T
    assert np.linalg.norm((_align(a) - _align(b))[m]) / np.linalg.norm(b[m]) <= 1e-4
