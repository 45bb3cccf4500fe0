"""The batched uneven-slice workload (square grids 192..320, Q 16..64, calibration 24..40,
ellipsoidal radius 3, f = 4): a batch of its extreme shapes must equal the single-plan path
item by item, and the largest items are checked against the FP64 oracle on sampled outputs
(the oracle's naive per-pixel G(x) over all ~1800 null vectors is too slow for every pixel):
the nullspace split, G(x), the power-iteration vector and eigenvalue at sampled reduced
pixels, and the interpolation + normalisation of the reduced-grid vectors at every pixel."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import pisco_oracle as O
from paper_2302_13431_gb300.phantoms import make_case, uneven_slice_specs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU collection
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2302_13431_gb300 import _binding as B  # noqa: E402
from paper_2302_13431_gb300.estimator import PiscoBatch, PiscoEstimator  # noqa: E402

ALL = uneven_slice_specs(96)


def _pick():
    """The extremes of the 96 shapes: largest/smallest Q x grid, smallest/largest calibration."""
    by_cost = sorted(range(96), key=lambda i: ALL[i]["num_coils"] ** 2 * ALL[i]["grid"][0] ** 2)
    by_cal = sorted(range(96), key=lambda i: ALL[i]["calib_shape"][0])
    idx = []
    for i in (by_cost[-1], by_cost[0], by_cal[0], by_cal[-1], by_cost[48]):
        if i not in idx:
            idx.append(i)
    q48 = next(i for i in range(96) if ALL[i]["num_coils"] == 48 and i not in idx)
    return idx + [q48]


PICK = _pick()
_state = {}


def _batch(precision):
    if precision in _state:
        return _state[precision]
    specs = [dict(ALL[i], precision=precision) for i in PICK]
    cases = [make_case(sp["grid"], sp["num_coils"], sp["calib_shape"], seed=sp["data_seed"]) for sp in specs]
    calibs = [torch.from_numpy(c.calib).cuda() for c in cases]
    batch = PiscoBatch(specs)
    maps, eigs = batch.alloc_outputs()
    batch.estimate_into(calibs, maps, eigs)
    batch.estimate_into(calibs, maps, eigs)  # captured graph
    torch.cuda.synchronize()
    _state[precision] = (specs, cases, calibs, batch, maps, eigs)
    return _state[precision]


@pytest.mark.parametrize("precision", ["fp32", "tc_g_eig"])
def test_uneven_batch_equals_single_plans(precision):
    specs, cases, calibs, batch, maps, eigs = _batch(precision)
    assert all(s == B.PISCO_OK for s in batch.last_item_status), batch.last_item_status
    for i, sp in enumerate(specs):
        est = PiscoEstimator(sp["grid"], sp["calib_shape"], sp["num_coils"], sp["tau"], reduction=sp["reduction"],
                             iters=sp["iters"], precision=precision)
        m1, e1 = est(calibs[i])
        torch.cuda.synchronize()
        assert torch.equal(m1, maps[i]) and torch.equal(e1, eigs[i]), i
        est.close()


@pytest.mark.parametrize("which", [0, 5])
@pytest.mark.parametrize("precision", ["fp32", "tc_g_eig"])
def test_uneven_item_against_oracle_on_samples(which, precision):
    specs, cases, calibs, batch, maps, eigs = _batch(precision)
    sp, case = specs[which], cases[which]
    Q, grid, f = sp["num_coils"], sp["grid"], sp["reduction"]
    red = tuple(g // f for g in grid)
    lam = O.kernel_support((3, 3), "ellipsoid")
    L = lam.shape[0]
    C = O.calibration_matrix(case.calib, lam, rows="full")
    V_null, U_sig, _ = O.nullspace_svd(C, 0.05)
    stats = batch.item_stats(which)
    assert stats["signal_dim"] == U_sig.shape[1]
    # sampled reduced pixels: inside the eroded support and anywhere
    rng = np.random.default_rng(7)
    inner = ndimage.binary_erosion(np.abs(case.rho) > 0, iterations=2)[::f, ::f].reshape(-1)
    cand_in = np.flatnonzero(inner)
    idx = np.unique(np.concatenate([rng.choice(cand_in, 40, replace=False),
                                    rng.choice(red[0] * red[1], 24, replace=False)]))
    xs = O.grid_points(red)[idx]
    G = O.G_direct(V_null, lam, Q, xs)
    Gg = batch.debug_buffer(which, B.PISCO_BUF_G).cpu().numpy().reshape(-1, Q, Q)[idx]
    assert np.abs(Gg - G).max() / L <= 2e-5
    v0 = O.start_vectors(0, red[0] * red[1], Q)[idx]
    v_pi, lam_pi, _ = O.power_iteration(G, v0, sp["iters"], L)
    v_al = O.phase_align(v_pi, O.apodised_lowres(case.calib, xs))
    w = np.linalg.eigvalsh(G) / L
    gapped = (w[:, 1] - w[:, 0]) > 1e-3
    V = batch.debug_buffer(which, B.PISCO_BUF_V).cpu().numpy().reshape(Q, -1).T
    vs = V[idx]
    al = lambda v: v * np.exp(-1j * np.angle(v[:, :1]))  # noqa: E731
    sel = gapped & inner[idx]
    assert sel.sum() >= 10
    err = np.linalg.norm((al(vs) - al(v_al))[sel]) / np.linalg.norm(v_al[sel])
    assert err <= 1e-4, err
    e_gpu = eigs[which].cpu().numpy().reshape(-1)[idx]
    assert np.abs(e_gpu - lam_pi)[sel].max() <= 1e-5
    # interpolation + normalisation of the GPU's reduced-grid vectors, every pixel
    full = O.normalize_maps(O.sinc_interp(V.astype(np.complex128), red, grid))
    got = maps[which].cpu().numpy().reshape(Q, -1).T
    rel = np.linalg.norm(got - full) / np.linalg.norm(full)
    assert rel <= 1e-5, rel


# the launch configuration the autotuner picks for this workload on the GB300, and plain FP32
ROUTES = {
    "tuned": dict(precision="tc_g_eig", tc_splits=1, gemm_splits=2, gemm_tile=64, gram_df=True, tc_interp=True),
    "fp32": dict(precision="fp32"),
}


def _golden_signal_dims():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "uneven96_signal_dims.txt")
    rows = [ln.split() for ln in open(path) if not ln.startswith("#")]
    return {int(r[0]): int(r[4]) for r in rows}


@pytest.mark.parametrize("route", sorted(ROUTES))
def test_all_96_slices_succeed_with_the_oracle_signal_dimension(route):
    """Every slice of the 96-slice workload (R >= Q|Lambda| - 128 > Q - 1 for all of them, so no
    slice may report a rank failure) returns PISCO_OK from one batched call, and its nullspace split
    equals the FP64 oracle's (SVD of the explicit C, stored by tests/golden/make_uneven_signal_dims.py)."""
    k_ref = _golden_signal_dims()
    specs = [dict(sp, **ROUTES[route]) for sp in ALL]
    calibs = [torch.from_numpy(make_case(sp["grid"], sp["num_coils"], sp["calib_shape"], seed=sp["data_seed"]).calib).cuda()
              for sp in specs]
    batch = PiscoBatch(specs)
    maps, eigs = batch.alloc_outputs()
    for _ in range(2):  # eager, then captured graph
        batch.estimate_into(calibs, maps, eigs)
        torch.cuda.synchronize()
        st = list(batch.last_item_status)
        assert st == [B.PISCO_OK] * 96, {i: s for i, s in enumerate(st) if s != B.PISCO_OK}
    ks = [batch.item_stats(i)["signal_dim"] for i in range(96)]
    bad = {i: (ks[i], k_ref[i]) for i in range(96) if ks[i] != k_ref[i]}
    assert not bad, bad
    for i in range(96):
        assert bool(torch.isfinite(torch.view_as_real(maps[i])).all()), i
        assert batch.item_stats(i)["cert_margin"] > 0, i
    batch.close()
